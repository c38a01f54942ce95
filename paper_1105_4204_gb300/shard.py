"""Host-side sharding of the filter across ranks (one process per GPU).

The filter partitions without exchanging intermediates:

* a batch of independent images is split across ranks by estimated cost
  (largest first onto the least-loaded rank), each rank filtering its own
  images;
* one large image is split into horizontal strips; a rank reads its strip
  plus a read-only halo of the spatial support radius (clipped at the image
  border, where the clamp-to-edge extension then coincides with the image's
  own), filters that sub-image and keeps its strip's rows;
* the backward pass of a shared sigma_r needs one collective: the sum over
  ranks of their dL/dsigma_r.

Nothing here touches a GPU; the functions are plain index arithmetic and a
torch.distributed call.
"""
from __future__ import annotations

from dataclasses import dataclass


def image_cost(H: int, W: int, n_terms: int, radius: int) -> float:
    """Relative cost of one image: terms x pixels, with the halo overhead of
    a 64-wide tile."""
    return float(n_terms) * H * W * (64.0 + 2.0 * radius) / 64.0


def shard_images(costs, world: int):
    """Largest-cost-first assignment of images to ranks.  Returns, per rank,
    the sorted list of image indices.  Deterministic for equal costs."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


@dataclass(frozen=True)
class Strip:
    rank: int
    y0: int      # first output row owned by the rank
    y1: int      # one past the last owned row
    r0: int      # first input row read (halo included, clipped to the image)
    r1: int      # one past the last input row read

    @property
    def crop(self):
        """Rows of the filtered sub-image [r0, r1) that the rank keeps."""
        return self.y0 - self.r0, self.y1 - self.r0


def row_strips(H: int, world: int, halo: int):
    """Split H rows into `world` contiguous strips (sizes differ by at most
    one row) with read-only halos of `halo` rows, clipped to [0, H)."""
    if world < 1 or H < 1 or halo < 0:
        raise ValueError("bad strip arguments")
    base, extra = divmod(H, world)
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        y0, y1 = y, y + n
        out.append(Strip(r, y0, y1, max(0, y0 - halo), min(H, y1 + halo)))
        y = y1
    return out


def allreduce_sigma_grad(value: float, group=None) -> float:
    """Sum of every rank's dL/dsigma_r (the one collective of the backward)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
