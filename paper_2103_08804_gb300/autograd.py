"""log psi of the RBM as a differentiable torch operation (Sec. I, Sec. III).

RBMLogPsi.apply(ctx, params, spins) returns log psi(sigma) for each walker
(complex, [B]) from `rbm_logpsi`; its backward is the hand-written VJP
kernel `logpsi_backward`: for a real loss L with upstream gradient
g_s = dL/d conj(log psi_s) (PyTorch's convention for complex tensors), the
parameter gradient is dL/d conj(alpha_k) = sum_s g_s conj(O_k(s)), with
O_k(s) = d log psi_s / d alpha_k (log psi is holomorphic in alpha).

Both directions run in libchebrbm kernels; torch only provides the
autograd bookkeeping.
"""

import torch


class RBMLogPsi(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cr_ctx, params, spins):
        B = spins.shape[0]
        theta = torch.empty(B, cr_ctx.M, dtype=cr_ctx.cdtype, device=spins.device)
        lp = cr_ctx.rbm_logpsi(params.detach().contiguous(), spins, theta_out=theta)
        fctx.cr_ctx = cr_ctx
        fctx.save_for_backward(params, spins, theta)
        return lp

    @staticmethod
    def backward(fctx, grad_lp):
        params, spins, theta = fctx.saved_tensors
        c = fctx.cr_ctx
        T = torch.empty_like(theta)
        c.logderiv(params.detach().contiguous(), spins, theta, tanh_out=T)
        g = c.logpsi_backward(params.detach().contiguous(), spins, T,
                              grad_lp.to(c.cdtype).contiguous())
        return None, g, None


def logpsi(cr_ctx, params, spins):
    """Differentiable log psi: complex [B]."""
    return RBMLogPsi.apply(cr_ctx, params, spins)


def overlap_loss(cr_ctx, params, spins, logpsi0, R):
    """The self-normalised importance-sampled infidelity of the fit (Sec. III)
    on fixed samples s of |psi_0|^2 (logpsi0 = log psi_0(s), complex):
        L(alpha) = -log( |sum_s w_s R_s|^2 / (sum_s w_s |R_s|^2 sum_s w_s) ),
    w_s = |psi_alpha(s) / psi_0(s)|^2 and R_s = phi_s / psi_alpha(s), given the
    target ratio R0_s = phi_s / psi_0(s) as R.  At alpha = alpha_0 its gradient
    with respect to conj(alpha) is -(<O* R>/<R> - <O*>), the bracket of the
    natural-gradient force F."""
    lp = logpsi(cr_ctx, params, spins)
    d = lp - logpsi0.to(lp.dtype)                  # log psi_alpha - log psi_0
    w = torch.exp(2.0 * d.real)
    Ra = R * torch.exp(-d)                         # phi / psi_alpha
    num = torch.abs(torch.sum(w * Ra)) ** 2
    den = torch.sum(w * torch.abs(Ra) ** 2) * torch.sum(w)
    return -torch.log(num / den)
