"""One image's quadrant over P ranks: row strips and one all-to-all.

A quadrant with n = 2^K slope rows and W columns splits over P = 2^p ranks
(P <= 8, P <= n) by the rows of the (transposed, for Q2/Q3) image:

1. rank r transforms its strip, image rows [r*n_s, (r+1)*n_s) with
   n_s = n/P, through the first K - p butterfly levels: the strip's own
   quadrant padded to n_s rows on the whole image's width W
   (fht_forward_padded), n_s x W;
2. one all-to-all: rank b receives, from every strip, the n_s/P rows
   tau in [b*n_s/P, (b+1)*n_s/P) (n*W/P^2 elements per pair);
3. rank b runs the last p levels on them (fht_merge_strips) and holds the
   quadrant's slope rows [b*n/P, (b+1)*n/P), bit for bit what one GPU
   computes: every output slope tau*P + c is the P-row transform of the
   strips' rows tau, row r read sheared by sigma*tau*r (the pass identity of
   the recursion), with the same additions in the same order.

The exchange is torch.distributed's all_to_all_single (NCCL between GPUs).
The two level steps are arguments, so that the same orchestration runs with
other implementations of them (the CPU test runs it on gloo ranks).
"""

from __future__ import annotations

import torch

import paper_1811_06378_gb300 as fht


class ShardPlan:
    """Geometry of quadrant q of an h x w image split over `ranks` ranks."""

    def __init__(self, h: int, w: int, q: int, ranks: int):
        if ranks not in (1, 2, 4, 8):
            raise ValueError("ranks must be 1, 2, 4 or 8")
        self.h, self.w, self.q, self.ranks = h, w, q, ranks
        self.n, self.W = fht.query_shape(h, w, q)
        if self.n % (ranks * ranks) and ranks > 1:
            raise ValueError(f"{ranks} ranks need n = {self.n} divisible by {ranks * ranks}")
        self.n_s = self.n // ranks             # strip rows, levels K - log2(ranks)
        self.block = self.n_s // ranks          # level rows per (strip, owner) pair
        self.rows_img = w if q >= 2 else h      # rows of the (transposed) image

    def strip(self, rank: int) -> tuple[int, int]:
        """(first, end) rows of the (transposed) image in rank's strip, cut to
        the image (end <= first for an empty strip)."""
        lo = rank * self.n_s
        return lo, min(lo + self.n_s, self.rows_img)

    def strip_of(self, img: torch.Tensor, rank: int) -> torch.Tensor:
        """Rank's strip of a whole image (a view): rows for Q0/Q1, columns
        for Q2/Q3."""
        lo, hi = self.strip(rank)
        hi = max(hi, lo)
        return img[:, lo:hi] if self.q >= 2 else img[lo:hi]

    def slopes(self, rank: int) -> tuple[int, int]:
        """(t_lo, t_hi) of the output slope rows rank holds."""
        per = self.n // self.ranks
        return rank * per, (rank + 1) * per - 1

    def exchange_elements(self) -> int:
        """Elements one rank sends to another in the all-to-all."""
        return self.block * self.W


def local_levels_gpu(strip: torch.Tensor, plan: ShardPlan, acc: torch.dtype) -> torch.Tensor:
    """Step 1 on the GPU: the strip's first K - log2(P) levels, (n_s, W)."""
    return fht.forward_padded(strip, plan.q, plan.n_s, plan.W, acc=acc)


def merge_levels_gpu(parts: torch.Tensor, plan: ShardPlan, rank: int) -> torch.Tensor:
    """Step 3 on the GPU: parts (P, n_s/P, W) from every strip -> this rank's
    (n/P, W) slope rows."""
    return fht.merge_strips(parts, plan.q, rank * plan.block)


def forward_sharded(strip: torch.Tensor, plan: ShardPlan, rank: int, group=None,
                    acc: torch.dtype = torch.int32, local=local_levels_gpu,
                    merge=merge_levels_gpu) -> torch.Tensor:
    """This rank's slope rows plan.slopes(rank) of the quadrant, from its strip
    (plan.strip_of(image, rank)), over the ranks of `group` (the default
    process group when None; nothing is exchanged for one rank)."""
    L = local(strip, plan, acc)                        # (n_s, W)
    if plan.ranks == 1:
        return merge(L.reshape(1, plan.n_s, plan.W), plan, rank)
    import torch.distributed as dist
    send = L.reshape(plan.ranks, plan.block, plan.W).contiguous()
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)    # recv[p] = strip p's rows of this block
    return merge(recv, plan, rank)                     # (n/P, W)
