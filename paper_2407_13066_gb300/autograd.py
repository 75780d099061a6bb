"""torch.autograd.Function wrappers: differentiation through the operator.

F is linear, so its Jacobian is F itself and the vector-Jacobian product of
d = F m is F* applied to the incoming gradient (the adjoint of Sec. 3.4,
real data so F* = F^T).  Each wrapper calls the library's hand-written
kernels in both directions:

    apply_F(op, m)              forward btt_matvec,  backward btt_adjoint
    apply_Fadj(op, d)           forward btt_adjoint, backward btt_matvec
    apply_H(op, m, gamma_inv)   forward btt_hessian, backward btt_hessian
                                (F* Gamma^-1 F is self-adjoint)

Gradients flow to the vectors only; the operator and gamma_inv are treated
as constants.
"""
import torch


class _ApplyF(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op):
        ctx.op = op
        return op.matvec(m.contiguous())

    @staticmethod
    def backward(ctx, grad_d):
        return ctx.op.adjoint(grad_d.contiguous()), None


class _ApplyFadj(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, op):
        ctx.op = op
        return op.adjoint(d.contiguous())

    @staticmethod
    def backward(ctx, grad_m):
        return ctx.op.matvec(grad_m.contiguous()), None


class _ApplyH(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op, gamma_inv):
        ctx.op = op
        ctx.gamma_inv = gamma_inv
        return op.hessian(m.contiguous(), gamma_inv)

    @staticmethod
    def backward(ctx, grad_y):
        return ctx.op.hessian(grad_y.contiguous(), ctx.gamma_inv), None, None


def apply_F(op, m):
    """d = F m, differentiable in m (backward = F*)."""
    return _ApplyF.apply(m, op)


def apply_Fadj(op, d):
    """m = F* d, differentiable in d (backward = F)."""
    return _ApplyFadj.apply(d, op)


def apply_H(op, m, gamma_inv=None):
    """y = F* Gamma^-1 F m, differentiable in m (backward = the same Hessian)."""
    return _ApplyH.apply(m, op, gamma_inv)
