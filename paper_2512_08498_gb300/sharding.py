"""One batch of views sharded over ranks, one process per GPU.

The per-keyframe optimisation renders every camera of the keyframe window
against the same Gaussians (Sec. 3.3 optimises the window's cameras jointly).
Across GPUs the batch splits by views: every rank holds a replica of the
Gaussians and runs the whole rasterization path (projection, lists, sort,
compositing and their adjoints) for a contiguous block of the views.  Its
images, losses and pose gradients stay local.  The Gaussian parameter
gradients of the batch are the sum of the ranks' gradients, and one
all-reduce (sum) of one flat buffer per iteration forms it: 4 (3 + 3 + 4 + 1
+ 3 K) bytes per Gaussian, 236 B at SH degree 3.  Nothing else is exchanged.

The functions here are host logic only (which views a rank renders, where
its gradients live, the one collective); the rendering is the library's.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch


def shard_bounds(pixels: Sequence[int], world: int) -> List[int]:
    """Contiguous blocks of views with about equal pixel counts: rank r
    renders views [b[r], b[r + 1]).  A view goes to the rank whose share of
    the cumulative pixel count holds the view's midpoint; ranks may get no
    view when there are fewer views than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    total = float(sum(int(p) for p in pixels))
    mids, c = [], 0.0
    for p in pixels:
        mids.append(c + 0.5 * float(p))
        c += float(p)
    bounds = [0]
    for r in range(1, world):
        cut = total * r / world
        bounds.append(sum(1 for m in mids if m < cut))
    bounds.append(len(pixels))
    return bounds


def shard_views(views: Sequence, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of the views rank renders (see shard_bounds)."""
    b = shard_bounds([int(v.width) * int(v.height) for v in views], world)
    return b[rank], b[rank + 1]


class GradBuffer:
    """The five parameter-gradient tensors of n Gaussians at SH degree
    `degree` as views of one flat float32 buffer, so that one all-reduce
    covers them.  Quaternions come first: their rows start 16-byte aligned,
    as the library requires."""

    def __init__(self, n: int, degree: int, device, dtype=torch.float32):
        k = (degree + 1) ** 2
        self.n, self.k = n, k
        sizes = [4 * n, 3 * n, 3 * n, n, 3 * k * n]
        self.flat = torch.zeros(sum(sizes), device=device, dtype=dtype)
        parts, o = [], 0
        for s in sizes:
            parts.append(self.flat[o:o + s])
            o += s
        self.quats = parts[0].view(n, 4)
        self.means = parts[1].view(n, 3)
        self.log_scales = parts[2].view(n, 3)
        self.opacity_logits = parts[3]
        self.sh = parts[4].view(n, k, 3)

    def tensors(self):
        """In the library's parameter order: means, log-scales, quaternions,
        opacity logits, SH."""
        return self.means, self.log_scales, self.quats, self.opacity_logits, self.sh

    def bytes_per_gaussian(self) -> int:
        return self.flat.element_size() * self.flat.numel() // max(self.n, 1)


def allreduce_grads(buf: GradBuffer, group=None) -> None:
    """Sum the ranks' parameter gradients in place: the one exchange of a
    view-sharded iteration.  On the current stream (NCCL) or the host
    (gloo)."""
    if torch.distributed.is_initialized() and torch.distributed.get_world_size(group) > 1:
        torch.distributed.all_reduce(buf.flat, op=torch.distributed.ReduceOp.SUM, group=group)
