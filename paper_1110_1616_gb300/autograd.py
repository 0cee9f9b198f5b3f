"""torch.autograd integration of the discrete adjoint: the coarse steps of a
context as a differentiable function of the packed initial state.

    u_final = advance(ctx, u0, dts, ckpt_every)

u0 and u_final are float64 CUDA tensors holding all 8 packed fields (the
amrmhd_backward layout). The forward runs amrmhd_step_dt_ckpt with the fixed
dt0 sequence dts (dt is not differentiated), keeping a checkpoint every
ckpt_every coarse steps; the backward differentiates that recorded forward
(amrmhd_backward_recorded: each segment recomputed from its checkpoint) while
the context still holds its final state, else it reloads u0 and calls
amrmhd_backward (forward pass, then the same sweep). Every step of both passes
runs in the library's CUDA kernels.
"""
import torch

from . import amrmhd as A


class AdvanceFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0, ctx, dts, ckpt_every):
        if not u0.is_cuda or u0.dtype != torch.float64:
            raise TypeError("u0 must be a float64 CUDA tensor")
        u0 = u0.contiguous()
        out = torch.empty_like(u0)
        # the library runs on its own stream: order it after torch's work and back
        torch.cuda.synchronize()
        ctx.load_packed_all(u0)
        ctx.step_dt_ckpt(dts, int(ckpt_every))
        ctx.read_packed_all(out)
        torch.cuda.synchronize()
        fctx.save_for_backward(u0)
        fctx.amr = ctx
        fctx.dts = list(dts)
        fctx.ckpt = int(ckpt_every)
        return out

    @staticmethod
    def backward(fctx, g):
        (u0,) = fctx.saved_tensors
        ctx = fctx.amr
        g = g.contiguous().to(torch.float64)
        g0 = torch.empty_like(u0)
        torch.cuda.synchronize()
        if not ctx.backward_recorded(g, g0):
            ctx.load_packed_all(u0)
            ctx.backward(fctx.dts, g, g0, fctx.ckpt)
        torch.cuda.synchronize()
        return g0, None, None, None


def advance(ctx: "A.Context", u0: torch.Tensor, dts, ckpt_every: int = 20) -> torch.Tensor:
    """Differentiable len(dts) coarse steps of ctx from the packed state u0."""
    return AdvanceFunction.apply(u0, ctx, dts, ckpt_every)


def velocity_gradient(u0: torch.Tensor, g0: torch.Tensor, ncells: int) -> torch.Tensor:
    """dL/dv0 (3 packed cell fields vx, vy, vz) from the packed initial state u0
    and dL/dU0 = the backward's output, with rho, p and B held
    (amrmhd_grad_velocity); ncells = the packed count of one cell field."""
    gv = torch.empty(3 * ncells, dtype=torch.float64, device=u0.device)
    torch.cuda.synchronize()
    st = A.lib().amrmhd_grad_velocity(int(ncells), A.C.c_void_p(u0.data_ptr()), A.C.c_void_p(g0.data_ptr()),
                                      A.C.c_void_p(gv.data_ptr()), None)
    if st != 0:
        raise RuntimeError("amrmhd_grad_velocity failed: status %d" % st)
    torch.cuda.synchronize()
    return gv
