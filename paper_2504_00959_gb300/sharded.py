"""One dirty image from measurements split across processes (one GPU each).

The imaging operator is linear in the visibilities (Eq. 3, FFT, Eq. 1), so
disjoint shards of the measurements image independently; the only exchange is
the sum of the partial images.  Each rank's image is normalised by its own
weight sum W_r, so the whole image is  I = sum_r W_r I_r / sum_r W_r  (grid
correction and the n factor are per-pixel factors common to all ranks).  This
is one all-reduce of n^2 values and one of a scalar -- instead of the
per-sector reduce of the w-plane grid the paper performs (Sec. 2.2), which
moves nw times more data.

Uniform weighting needs the density of all shards before gridding and is not
offered here.
"""
import torch
import torch.distributed as dist


def combine_images(image, sum_w, group=None):
    """Sum the partial images of all ranks, each normalised by its own weight
    sum ``sum_w`` (a float), into the image of all measurements.  Returns a
    new tensor of the same dtype on the same device."""
    w = torch.tensor([float(sum_w)], dtype=torch.float64, device=image.device)
    num = image * float(sum_w)
    dist.all_reduce(num, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    total = float(w.item())
    return num / total if total != 0.0 else torch.zeros_like(num)


class ShardedImager:
    """An ``Imager`` per rank over that rank's share of the measurements, and
    the combined image.  ``params`` must not ask for uniform weighting."""

    def __init__(self, params, device=None, group=None):
        from . import Imager, UNIFORM_WEIGHT
        if int(params.get("flags", 0)) & UNIFORM_WEIGHT:
            raise ValueError("uniform weighting needs the density of every shard; not available when sharded")
        self.imager = Imager(params, device=device)
        self.group = group

    def grid(self, vis, u, v, w, wt=None):
        self.imager.grid(vis, u, v, w, wt)

    def reset(self):
        self.imager.reset()

    def image(self):
        img = self.imager.image()
        sw = self.imager.stats()["sum_weights"]
        return combine_images(img, sw, self.group)

    def close(self):
        self.imager.close()
