"""``torch.autograd.Function`` over the FP32 fitness kernels of libpsso.so
(psso_fitness_forward_ws / psso_fitness_backward_ws): f = fitness(X) for the
rows of a CUDA float32 tensor, differentiable with respect to X.  The rotated
functions' products z = M (x - o) and M^T df/dz run on the tensor cores, in a
workspace taken from torch's caching allocator.

The tensors are plumbing only: both passes run in the library's kernels, on
torch's current CUDA stream.
"""
from __future__ import annotations

import torch

from . import FN, psso_fitness_backward_ws, psso_fitness_forward_ws, psso_fitness_workspace_size


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def _workspace(fn, N, D, device):
    n = psso_fitness_workspace_size(fn, N, D)
    if n == 0:
        return None, 0
    # the caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(n, dtype=torch.uint8, device=device), n


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
        ws, nws = _workspace(fn, N, D, X.device)
        psso_fitness_forward_ws(fn, N, D, X.data_ptr(), shift.data_ptr(), _ptr(weights),
                                _ptr(rotation), f.data_ptr(), _ptr(ws), nws, _stream(X.device))
        ctx.save_for_backward(X, shift, weights, rotation)
        ctx.fn = fn
        return f

    @staticmethod
    def backward(ctx, grad_f):
        X, shift, weights, rotation = ctx.saved_tensors
        N, D = X.shape
        grad_f = grad_f.to(torch.float32).contiguous()
        gX = torch.empty_like(X)
        ws, nws = _workspace(ctx.fn, N, D, X.device)
        psso_fitness_backward_ws(ctx.fn, N, D, X.data_ptr(), shift.data_ptr(), _ptr(weights),
                                 _ptr(rotation), grad_f.data_ptr(), gX.data_ptr(), _ptr(ws), nws,
                                 _stream(X.device))
        return gX, None, None, None, None


def fitness(X, fn, shift, weights=None, rotation=None):
    """Differentiable FP32 fitness of the rows of X (N x D, float32, CUDA)."""
    return Fitness.apply(X, fn, shift, weights, rotation)
