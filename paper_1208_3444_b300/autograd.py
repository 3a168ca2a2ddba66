"""torch.autograd bindings of the library's hand-written derivative kernels.

``AllPairsForce.apply(x, m, sim)`` returns the comoving acceleration of Eq. 1
(``colatus_forces``); its backward is the VJP kernel (``colatus_force_vjp``).

``Trajectory.apply(x0, v0, m, sim, dt, nsteps, checkpoint_every)`` runs the
KDK leapfrog with Hubble drag (``colatus_adjoint_forward``) and returns the
final (x, v); its backward is the checkpointed discrete adjoint
(``colatus_adjoint_backward``).  ``sim`` is a ``binding.Simulation`` whose
configuration (precision, G, cosmology, eps, a at the start) is used as is;
its state is overwritten.  Tensors live on the simulation's CUDA device, in
float32 or float64.
"""
import torch

from . import binding as B


class AllPairsForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, m, sim):
        x = x.detach().contiguous()
        m = m.detach().contiguous()
        sim.set_masses(m)
        sim.set_state(x)
        acc = torch.empty_like(x)
        sim.forces(acc)
        ctx.sim = sim
        ctx.save_for_backward(x, m)
        return acc

    @staticmethod
    def backward(ctx, gacc):
        sim = ctx.sim
        x, m = ctx.saved_tensors
        sim.set_masses(m)
        sim.set_state(x)
        gx = torch.empty_like(x)
        gm = torch.empty_like(m)
        B.colatus_force_vjp(sim.h, gacc.contiguous(), gx, gm)
        return gx, gm, None


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, sim, dt, nsteps, checkpoint_every):
        sim.set_masses(m.detach().contiguous())
        sim.set_state(x0.detach().contiguous(), v0.detach().contiguous())
        sim.adjoint_forward(dt, nsteps, checkpoint_every)
        xT = torch.empty_like(x0)
        vT = torch.empty_like(v0)
        B.colatus_get_state(sim.h, xT, vT)
        ctx.sim = sim
        ctx.m_like = m
        return xT, vT

    @staticmethod
    def backward(ctx, gxT, gvT):
        sim = ctx.sim
        gx0 = torch.empty_like(gxT)
        gv0 = torch.empty_like(gvT)
        gm = torch.empty_like(ctx.m_like)
        B.colatus_adjoint_backward(sim.h, gxT.contiguous(), gvT.contiguous(), None, gx0, gv0, gm)
        return gx0, gv0, gm, None, None, None, None
