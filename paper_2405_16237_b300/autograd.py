"""torch.autograd.Function around the library's training forward and its
hand-written adjoint (nbvh_forward_train / nbvh_backward): gradients of the
raw MLP outputs of a batch of segments with respect to the hash table and the
MLP parameters. Argument marshalling only; both directions run in the
library's kernels."""
from __future__ import annotations

import torch

from . import nbvh as B


class NBVHQueryFn(torch.autograd.Function):
    """raw = NBVHQueryFn.apply(table, mlp, desc, rays, leaf, t0, t1, workspace)

    table: FP32 [entries, F] (also read by the kernels), mlp: FP32 parameters;
    rays/leaf/t0/t1 describe one segment per ray (leaf < 0: no segment).
    Returns raw outputs [n, n_out]; backward returns dL/dtable and dL/dmlp."""

    @staticmethod
    def forward(ctx, table, mlp, desc, rays, leaf, t0, t1, workspace):
        raw = B.forward_train(desc, table, mlp, rays, leaf, t0, t1, workspace)
        ctx.desc = desc
        ctx.rays = rays
        ctx.save_for_backward(table, mlp, leaf, t0, t1, workspace)
        return raw

    @staticmethod
    def backward(ctx, grad_raw):
        table, mlp, leaf, t0, t1, workspace = ctx.saved_tensors
        g_table = torch.zeros_like(table, dtype=torch.float32)
        g_mlp = torch.zeros_like(mlp)
        B.backward(ctx.desc, table, mlp, ctx.rays, leaf, t0, t1, workspace, g_table, g_mlp,
                   grad_out=grad_raw.contiguous().float())
        return g_table, g_mlp, None, None, None, None, None, None
