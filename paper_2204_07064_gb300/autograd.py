"""torch.autograd.Function over the streamed model (chunked, checkpointed).

Forward: the input is streamed chunk by chunk through the library
(cc_process_batch_strided); before each chunk the streams' cached state (the
kept rows of every ring, not the whole arena slot) is copied into a device
checkpoint by one kernel (cc_snapshot_batch), so memory grows with the number
of chunks times the per-stream cache, not with the signal's activations.
Backward: the checkpoints are restored in reverse order and the library's
hand-written backward (cc_backward_chunk) recomputes each chunk and
propagates the adjoints, carrying the cache adjoint from chunk to chunk;
weight and bias gradients accumulate in a Grads object (the input's gradient
is computed only when the input requires it).  After the backward
the streams are back in the state the forward left them in.
"""
from __future__ import annotations

import torch

from . import api


class StreamedRunner:
    """A model (FP32, or BF16/FP16 created with fuse_units=False: the forward
    then runs on the tensor cores and the gradients are those of that
    arithmetic), its streams, gradient buffers and the chunk length."""

    def __init__(self, model, params, streams, chunk_steps):
        self.model = model
        self.streams = list(streams)
        self.grads = api.Grads(model, params)
        io = model.io
        self.in_chunk = chunk_steps * io["in_per_step"]
        self.out_chunk = chunk_steps * io["out_per_step"]
        self.io = io
        self.anchor = None

    def weights_anchor(self, device):
        """A zero-size tensor that requires a gradient and stands for the
        model's weights in the autograd graph (their gradients land in
        self.grads), so that the backward runs when only they need one."""
        if self.anchor is None or self.anchor.device != device:
            self.anchor = torch.zeros(0, device=device, requires_grad=True)
        return self.anchor


class _Streamed(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, anchor, runner):
        count, n_in, cin = x.shape
        io = runner.io
        if n_in % runner.in_chunk:
            raise ValueError("input length must be a whole number of chunks")
        chunks = n_in // runner.in_chunk
        nb = api.snapshot_bytes(runner.model)
        ckpt = torch.empty((chunks + 1, count * nb), dtype=torch.uint8, device=x.device)
        y = torch.empty((count, chunks * runner.out_chunk, io["out_channels"]), dtype=torch.float32,
                        device=x.device)
        xs = x.detach().contiguous()
        for c in range(chunks):
            api.snapshot_batch(runner.model, runner.streams, ckpt[c])
            xc = xs[:, c * runner.in_chunk:(c + 1) * runner.in_chunk].contiguous()
            yc = torch.empty((count, runner.out_chunk, io["out_channels"]), dtype=torch.float32, device=x.device)
            runner.model.process_batch(runner.streams, xc, yc)
            y[:, c * runner.out_chunk:(c + 1) * runner.out_chunk] = yc
        api.snapshot_batch(runner.model, runner.streams, ckpt[chunks])
        ctx.save_for_backward(xs, ckpt)
        ctx.runner = runner
        ctx.chunks = chunks
        return y

    @staticmethod
    def backward(ctx, gy):
        xs, ckpt = ctx.saved_tensors
        runner = ctx.runner
        gy = gy.contiguous()
        want_gx = ctx.needs_input_grad[0]
        gx = torch.zeros_like(xs) if want_gx else None
        runner.grads.begin(runner.streams)
        for c in reversed(range(ctx.chunks)):
            api.restore_batch(runner.model, runner.streams, ckpt[c])
            xc = xs[:, c * runner.in_chunk:(c + 1) * runner.in_chunk].contiguous()
            gyc = gy[:, c * runner.out_chunk:(c + 1) * runner.out_chunk].contiguous()
            gxc = torch.empty_like(xc) if want_gx else None
            runner.grads.chunk(runner.streams, xc, gyc, gxc)
            if want_gx:
                gx[:, c * runner.in_chunk:(c + 1) * runner.in_chunk] = gxc
        api.restore_batch(runner.model, runner.streams, ckpt[ctx.chunks])
        return gx, None, None


def streamed(x, runner):
    """y = the streamed model applied to x [count][n_in][C_in]; y.backward()
    accumulates the weight and bias gradients in runner.grads, and x's
    gradient when x requires one."""
    return _Streamed.apply(x, runner.weights_anchor(x.device), runner)
