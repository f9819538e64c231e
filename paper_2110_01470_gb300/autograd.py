"""``torch.autograd.Function`` over the FP32 fitness kernels of libpsso.so
(psso_fitness_forward / psso_fitness_backward): f = fitness(X) for the rows
of a CUDA float32 tensor, differentiable with respect to X.

The tensors are plumbing only: both passes run in the library's kernels, on
torch's current CUDA stream.
"""
from __future__ import annotations

import torch

from . import FN, psso_fitness_backward, psso_fitness_forward


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


class Fitness(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, fn, shift, weights=None, rotation=None):
        if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
            raise TypeError("X must be a 2-D float32 CUDA tensor")
        X = X.contiguous()
        N, D = X.shape
        shift = shift.to(X.device, torch.float32).contiguous()
        weights = None if weights is None else weights.to(X.device, torch.float32).contiguous()
        rotation = None if rotation is None else rotation.to(X.device, torch.float32).contiguous()
        f = torch.empty(N, device=X.device, dtype=torch.float32)
        fn = FN[fn] if isinstance(fn, str) else int(fn)
        psso_fitness_forward(fn, N, D, X.data_ptr(), shift.data_ptr(), _ptr(weights), _ptr(rotation),
                             f.data_ptr(), _stream(X.device))
        ctx.save_for_backward(X, shift, weights, rotation)
        ctx.fn = fn
        return f

    @staticmethod
    def backward(ctx, grad_f):
        X, shift, weights, rotation = ctx.saved_tensors
        N, D = X.shape
        grad_f = grad_f.to(torch.float32).contiguous()
        gX = torch.empty_like(X)
        psso_fitness_backward(ctx.fn, N, D, X.data_ptr(), shift.data_ptr(), _ptr(weights),
                              _ptr(rotation), grad_f.data_ptr(), gX.data_ptr(), _stream(X.device))
        return gX, None, None, None, None


def fitness(X, fn, shift, weights=None, rotation=None):
    """Differentiable FP32 fitness of the rows of X (N x D, float32, CUDA)."""
    return Fitness.apply(X, fn, shift, weights, rotation)
