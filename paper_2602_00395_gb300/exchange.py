"""Data-parallel exchange of the gradient and Hutchinson buffers over views.

Sec. 4.1 defines g = (1/m) (M/|S1|) sum_{i in S1} J_i^T f_i and the Hutchinson
diagonal with the same (1/m) scaling.  When a step's views are split across
ranks, each rank's gs_raster_bwd normalises by its own residual count m_r, so the
global buffers are the m_r/m-weighted sums

    g = sum_r (m_r / m) g_r,      hz = sum_r (m_r / m) hz_r,      m = sum_r m_r,

after which every rank applies the identical, deterministic gs_tr_update.  The
exchange is one all-reduce (sum) per buffer; with one rank it does nothing.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class GradExchange:
    def __init__(self, group=None):
        self.group = group

    def world(self) -> int:
        return dist.get_world_size(self.group) if dist.is_available() and dist.is_initialized() else 1

    def __call__(self, m_local: float, *buffers: torch.Tensor) -> float:
        """Reweight and sum `buffers` in place across ranks; returns the global m."""
        if self.world() == 1:
            return float(m_local)
        m = torch.tensor([float(m_local)], dtype=torch.float64, device=buffers[0].device)
        dist.all_reduce(m, group=self.group)
        m_total = float(m.item())
        w = float(m_local) / m_total
        for b in buffers:
            if b is None:
                continue
            b.mul_(w)
            dist.all_reduce(b, group=self.group)
        return m_total
