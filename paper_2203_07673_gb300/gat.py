"""Multi-head graph-attention layer, forward (Sec. VI-E, GAT workload).

A layer maps node features X (n x r_in) to heads * rh output features:
    H = X W                      (one dense GEMM; cuBLAS through torch.matmul)
    f = per-head H a_l, g = per-head H a_r     (fmm_gat_project)
    out_i = sum_j softmax_j(LeakyReLU(s_ij (f_i + g_j))) H_j   per head
                                 (fmm_gat_forward: one gather pass per row)
The paper runs this forward pass with random weights to measure the sparse
work; so does bench.py --gat.
"""
from __future__ import annotations

import torch

from . import fmm


def gat_layer(plan: fmm.Plan, X: torch.Tensor, W: torch.Tensor, a_l: torch.Tensor,
              a_r: torch.Tensor, heads: int, slope: float = 0.2, vals=None):
    """One forward pass; returns (out, H).  plan.r must equal heads * rh =
    W.shape[1]; H is computed in float32 and cast to the plan's dtype."""
    H = X @ W
    f = fmm.gat_project(H, a_l, heads)
    g = fmm.gat_project(H, a_r, heads)
    Hp = H if plan.dtype == torch.float32 else H.to(plan.dtype)
    out = fmm.gat_forward(plan, heads, vals, f, g, Hp.contiguous(), slope)
    return out, H
