"""torch.autograd.Function over the forward modelling operator.

forward:  receiver traces d = F(m) via wave_fwd, checkpointing the wavefield
          every `ckpt_every` steps;
backward: dL/dm = wave_grad(residual = dL/dd), which recomputes each segment
          from its checkpoint and runs the adjoint sweep with the imaging
          condition.  Only m is differentiated.
"""
import torch

from . import wave


class WaveModeling(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, grid, damp, src_xyz, src_traces, rec_xyz, ckpt_every=50, tuning=None):
        rec, _, ckpt, _ = wave.fwd(grid, m.detach().contiguous(), damp, src_xyz, src_traces, rec_xyz,
                                   tuning=tuning, ckpt_every=ckpt_every)
        ctx.save_for_backward(m.detach(), damp, src_traces, ckpt)
        ctx.grid = grid
        ctx.src_xyz = src_xyz
        ctx.rec_xyz = rec_xyz
        ctx.ckpt_every = ckpt_every
        ctx.tuning = tuning
        return rec

    @staticmethod
    def backward(ctx, grad_rec):
        m, damp, src_traces, ckpt = ctx.saved_tensors
        g, _ = wave.grad(ctx.grid, m.contiguous(), damp, ctx.src_xyz, src_traces, ctx.rec_xyz,
                         grad_rec.contiguous(), ckpt, ctx.ckpt_every, tuning=ctx.tuning)
        return g, None, None, None, None, None, None, None


def modeling(m, grid, damp, src_xyz, src_traces, rec_xyz, ckpt_every=50, tuning=None):
    """Receiver traces as a differentiable function of m."""
    return WaveModeling.apply(m, grid, damp, src_xyz, src_traces, rec_xyz, ckpt_every, tuning)
