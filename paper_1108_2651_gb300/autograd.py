"""torch.autograd.Function over the library's forward run and hand-written adjoint.

receiver_traces(eps, problem, ...) returns the receiver traces [nrec, nsteps]
of a run from zero initial fields in the medium eps_r = eps (uniform mu);
its backward calls lbem_adjoint, the reverse-time adjoint stream-collide
kernel with checkpoint-and-recompute every `checkpoint_every` steps and the
gradient accumulated over time steps in FP64.  Any loss of the traces can be
differentiated, e.g. the L2 misfit 1/2 sum (traces - obs)^2.
"""
import numpy as np
import torch

from . import lbem


class _Traces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, solver, site, comp, amp, rec_site, rec_comp, nsteps, every):
        h = solver.h
        e = eps.detach().to(torch.float32).contiguous().view(-1)
        lbem.lbem_set_medium(h, e)
        lbem.lbem_set_sources(h, site, comp, amp)
        lbem.lbem_set_receivers(h, rec_site, rec_comp, nsteps)
        lbem.lbem_set_fields(h)
        lbem.lbem_forward_record(h, nsteps, every)
        nrec = len(rec_site)
        out = torch.empty(max(nrec * nsteps, 1), dtype=torch.float32, device=eps.device)
        if nrec:
            lbem.lbem_traces(h, out)
        ctx.solver = solver
        ctx.shape = eps.shape
        return out[: nrec * nsteps].view(nrec, nsteps)

    @staticmethod
    def backward(ctx, gtr):
        h = ctx.solver.h
        g = gtr.detach().to(torch.float32).contiguous()
        grad = torch.empty(int(np.prod(ctx.shape)), dtype=torch.float32, device=gtr.device)
        lbem.lbem_adjoint(h, g.view(-1), grad)
        return grad.view(ctx.shape), None, None, None, None, None, None, None, None


def receiver_traces(eps, solver, problem, nsteps=None, checkpoint_every=100):
    """Differentiable receiver traces of `problem` (a workloads.Problem) in medium eps (torch CUDA tensor)."""
    nsteps = problem.nsteps if nsteps is None else nsteps
    return _Traces.apply(eps, solver, problem.src_site, problem.src_comp, problem.src_amp[:, :nsteps],
                         problem.rec_site, problem.rec_comp, nsteps, checkpoint_every)


def misfit(traces, obs):
    """L = 1/2 sum (traces - obs)^2, accumulated in FP64."""
    d = traces.double() - obs.double()
    return 0.5 * (d * d).sum()
