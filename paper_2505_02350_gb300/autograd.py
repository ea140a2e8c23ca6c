"""torch.autograd.Function around the forward (Eq. 3-26) and the adjoint (App. A).

``erbf_field(problem, p)`` returns Psi at the problem's binned training
points for the parameter tensor ``p`` (10 x cap, float32, on the problem's
device).  Its backward recomputes the basis values in the adjoint kernels --
nothing per pair is stored -- and returns dL/dp for any upstream gradient
dL/dPsi.  The neighbour lists are rebuilt for ``p`` on every forward.
"""
import torch

from . import _native as N


class ERBFField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, problem):
        if p.data_ptr() != problem.p.data_ptr():
            problem.p.copy_(p)
        problem.build_neighbors()
        problem.forward()
        ctx.problem = problem
        return problem.psi[:problem.n].clone()

    @staticmethod
    def backward(ctx, g_psi):
        pb = ctx.problem
        # serbf_backward returns d(sum_i err_i^2)/dp = sum_i 2 err_i dPsi_i/dp,
        # so err = g / 2 gives sum_i g_i dPsi_i/dp
        err = (0.5 * g_psi).contiguous().to(torch.float32)
        grad = torch.zeros_like(pb.grad)
        N.serbf_backward(pb.pts, pb.prm, pb.cfg, err, grad, pb.stats, pb.ws)
        m = pb.m()
        if m < grad.shape[1]:
            grad[:, m:] = 0
        return grad, None


def erbf_field(problem, p):
    return ERBFField.apply(p, problem)
