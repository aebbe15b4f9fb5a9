"""``torch.autograd.Function`` wrappers over the library's training calls.

Argument marshalling only: the forward and backward of every Function run in
the library's kernels (``gw_trainer_forward`` / ``gw_trainer_backward``,
``gw_band_loss`` / ``gw_band_loss_backward``, ``gw_whiten`` /
``gw_fir_backward``); PyTorch provides the tensors, the stream and the tape of
Functions.  Tensors must be CUDA float32.

    trainer = gwstream.gw_trainer_create(ctx, 21, B, L)
    y = DeepCleanFn.apply(x, params, trainer)       # params: raw FP32, requires_grad
    loss = BandLossFn.apply(strain, y, loss_fir)
    loss.backward()                                 # params.grad = dLoss/dparams
"""
from __future__ import annotations

import torch

from . import gwstream as G


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _f32(t):
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError("expected a CUDA float32 tensor")
    return t.contiguous()


class DeepCleanFn(torch.autograd.Function):
    """y_hat [B][L] = DeepClean(x [B][C][L]; raw params) with BatchNorm folded
    from its running statistics; backward gives dLoss/dparams (x gets none).
    One forward per trainer may be awaiting its backward at a time."""

    @staticmethod
    def forward(ctx, x, params, trainer):
        x, params = _f32(x), _f32(params)
        B, _, L = x.shape
        y = torch.empty(B, L, device=x.device, dtype=torch.float32)
        G.gw_trainer_forward(trainer, params.data_ptr(), x.data_ptr(), B, y.data_ptr(), _stream())
        ctx.trainer = trainer
        ctx.save_for_backward(params)
        return y

    @staticmethod
    def backward(ctx, dy):
        (params,) = ctx.saved_tensors
        dp = torch.empty_like(params)
        G.gw_trainer_backward(ctx.trainer, _f32(dy).data_ptr(), dp.data_ptr(), _stream())
        return None, dp, None


class BandLossFn(torch.autograd.Function):
    """Scalar loss (1/N) sum (g (*) (strain - y_hat))^2, valid mode."""

    @staticmethod
    def forward(ctx, strain, y_hat, fir):
        strain, y_hat = _f32(strain), _f32(y_hat)
        B, L = y_hat.shape
        K = G.gw_fir_ntaps(fir)
        loss = torch.empty((), device=y_hat.device, dtype=torch.float32)
        r = torch.empty(B, L - K + 1, device=y_hat.device, dtype=torch.float32)
        G.gw_band_loss(fir, strain.data_ptr(), y_hat.data_ptr(), B, L, loss.data_ptr(), r.data_ptr(), _stream())
        ctx.fir, ctx.shape = fir, (B, L)
        ctx.save_for_backward(r)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (r,) = ctx.saved_tensors
        B, L = ctx.shape
        dy = torch.empty(B, L, device=r.device, dtype=torch.float32)
        G.gw_band_loss_backward(ctx.fir, r.data_ptr(), B, L, _f32(dloss).data_ptr(), dy.data_ptr(), _stream())
        return None, dy, None


class FirFn(torch.autograd.Function):
    """Valid-mode FIR (whitening) y[b][c][n] = sum_k h[k] x[b][c][n + k]."""

    @staticmethod
    def forward(ctx, x, fir):
        x = _f32(x)
        B, C, L = x.shape
        K = G.gw_fir_ntaps(fir)
        y = torch.empty(B, C, L - K + 1, device=x.device, dtype=torch.float32)
        G.gw_whiten(fir, x.data_ptr(), B, C, L, y.data_ptr(), _stream())
        ctx.fir, ctx.shape = fir, (B, C, L)
        return y

    @staticmethod
    def backward(ctx, dy):
        B, C, L = ctx.shape
        dx = torch.empty(B, C, L, device=dy.device, dtype=torch.float32)
        G.gw_fir_backward(ctx.fir, _f32(dy).data_ptr(), B, C, L, dx.data_ptr(), _stream())
        return dx, None
