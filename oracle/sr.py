"""VMC estimators and the modified natural-gradient update (Sec. III).

With samples s drawn from |psi_s|^2 / <psi|psi> (or, in enumeration mode,
exact weights p_s = |psi_s|^2 / sum |psi|^2 over the whole S^z sector):

    S_kk' = <O_k* O_k'> - <O_k>* <O_k'>
    gamma = arccos sqrt( |<R>|^2 / <|R|^2> )
    F_k   = dgamma * gamma cot(gamma) * ( <O_k* R> / <R> - <O_k*> )

and the update solves sum_k' (S + lambda I)_kk' dalpha_k' = F_k, then sets
alpha <- alpha + dalpha.  Readings of points the paper leaves open:
  * the diagonal shift is additive, S + lambda I;
  * the argument of the arccos is clamped to <= 1 (sampling noise can push
    it above), and gamma cot gamma is taken as 1 when gamma < 1e-8;
  * the shifted system is solved by Cholesky (S + lambda I is Hermitian
    positive definite for lambda > 0), or by conjugate gradients, plain or
    with the Jacobi preconditioner diag(S) + lambda, from x = 0.
"""

import numpy as np
import scipy.linalg


def _mean(x, weights):
    if weights is None:
        return np.mean(x, axis=0)
    return np.tensordot(weights, x, axes=(0, 0))


def estimators(O, R, weights=None, with_OO=True):
    """The sample averages the update needs.

    O [B, P] complex log-derivatives, R [B] complex ratios, weights [B] (sum 1)
    or None for plain sample means.  with_OO=False leaves out <O* O^T> (P x P),
    for the matrix-free solve.
    """
    O = np.asarray(O, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    est = {
        "mR": _mean(R, weights),
        "mRR": _mean(np.abs(R) ** 2, weights).real,
        "Obar": _mean(O, weights),
        "OR": _mean(np.conj(O) * R[:, None], weights),
    }
    if with_OO:
        est["OO"] = (np.conj(O).T * (np.ones(len(R)) / len(R) if weights is None else weights)) @ O
    return est


def fubini_study_angle(mR, mRR):
    """gamma = arccos sqrt(|<R>|^2 / <|R|^2>), argument clamped to <= 1."""
    return float(np.arccos(np.sqrt(min(1.0, abs(mR) ** 2 / mRR))))


def gamma_cot_gamma(gamma):
    return 1.0 if gamma < 1e-8 else gamma / np.tan(gamma)


def force(est, dgamma):
    """F_k and gamma from the estimators."""
    gamma = fubini_study_angle(est["mR"], est["mRR"])
    c = dgamma * gamma_cot_gamma(gamma)
    F = c * (est["OR"] / est["mR"] - np.conj(est["Obar"]))
    return F, gamma


def qgt(est):
    """S = <O* O^T> - <O>* <O>^T  (the quantum geometric tensor, Sec. III)."""
    return est["OO"] - np.outer(np.conj(est["Obar"]), est["Obar"])


def shifted_solve(S, F, shift):
    """Solve (S + shift I) x = F by Cholesky."""
    A = S + shift * np.eye(S.shape[0])
    c = scipy.linalg.cho_factor(A, lower=True)
    return scipy.linalg.cho_solve(c, F)


def cg_solve(S, F, shift, maxit, tol, jacobi=False):
    """(S + shift I) x = F by conjugate gradients from x = 0 (Hestenes and
    Stiefel 1952), optionally with the Jacobi preconditioner diag(S) + shift.
    Stops when |r| <= tol |F| or after maxit iterations.  Returns (x, iterations)."""
    A = S + shift * np.eye(S.shape[0])
    d = np.real(np.diag(A)) if jacobi else np.ones(S.shape[0])
    return cg_solve_op(lambda v: A @ v, F, d, maxit, tol)


def cg_solve_op(apply, F, d, maxit, tol):
    """The same conjugate gradients with the operator given as a function,
    apply(v) = (S + shift I) v (the matrix-free form of Sec. III), and the
    preconditioner diagonal d (ones for plain CG).  Returns (x, iterations)."""
    x = np.zeros_like(F)
    r = F.copy()
    z = r / d
    p = z.copy()
    rz = np.vdot(r, z).real
    f2 = np.vdot(F, F).real
    it = 0
    if f2 == 0.0:
        return x, 0
    while it < maxit:
        Ap = apply(p)
        alpha = rz / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        if np.vdot(r, r).real <= tol * tol * f2:
            break
        z = r / d
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


def sv_matrix_free(O_blocks, v, shift):
    """(S + shift I) v = O^dag (O v) / B - Obar^* (Obar . v) + shift v from the
    log-derivatives given block by block (an iterable of [b, P] arrays whose
    rows are all the samples), without forming S."""
    acc = np.zeros(len(v), dtype=np.complex128)
    sumO = np.zeros(len(v), dtype=np.complex128)
    B = 0
    for O in O_blocks:
        acc += np.conj(O).T @ (O @ v)
        sumO += O.sum(axis=0)
        B += O.shape[0]
    Obar = sumO / B
    return acc / B - np.conj(Obar) * (Obar @ v) + shift * v


def sr_step(params, O, R, shift, dgamma, weights=None, solver="cholesky", cg_maxit=100,
            cg_tol=1e-6, jacobi=False):
    """One natural-gradient update.  Returns (new params, info dict).

    solver "cholesky": direct solve; "cg": cg_solve with the given options."""
    est = estimators(O, R, weights)
    F, gamma = force(est, dgamma)
    S = qgt(est)
    if solver == "cholesky":
        delta = shifted_solve(S, F, shift)
    else:
        delta, _ = cg_solve(S, F, shift, cg_maxit, cg_tol, jacobi)
    info = {"gamma": gamma, "mR": est["mR"], "mRR": est["mRR"], "F": F, "S": S,
            "delta": delta, "Obar": est["Obar"], "OR": est["OR"]}
    return np.asarray(params, dtype=np.complex128) + delta, info
