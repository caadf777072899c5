"""One dirty image on several GPUs (one process per GPU, torch.distributed).

Every step of the imaging operator is linear -- in the visibilities (Eq. 3,
the plane FFT, Eq. 1) and in the w-planes (Eq. 1 sums them) -- and the
finalisation (fftshift sign, 1 / weight sum, taper, n) is a per-pixel factor.
So images of disjoint shares of the work, normalised by the same weight sum,
add up to the image of everything, and the only exchange is one all-reduce
(sum) of the n^2 image -- instead of the reduce of the gridded w-planes of
every sector onto their owner that the paper performs (Sec. 2.2), which moves
nw times more data.  Two ways to share the work, both done by the library:

* ``mode="planes"`` (default): every rank takes all measurements and the
  w-planes [r nw / N, (r+1) nw / N) (``rick_set_plane_range``): the gridding,
  FFT and stacking split N ways, every rank's weight sum is already the total,
  and uniform weighting counts all measurements on every rank.
* ``mode="measurements"``: rank r grids its own share of the measurements;
  the ranks' weight sums are summed (an all-reduce of one scalar) and set on
  every rank (``rick_set_weight_sum``) before its image is made.  Uniform
  weighting would need the density of every shard first and is refused.

Python only marshals and calls the collectives.
"""
import torch
import torch.distributed as dist


def plane_share(nw, rank, world):
    """The w-planes [k0, k1) of rank `rank` out of `world` (contiguous, sizes
    differing by at most one)."""
    if world > nw:
        raise ValueError(f"{world} ranks cannot share {nw} w-planes")
    return (rank * nw) // world, ((rank + 1) * nw) // world


def _all_reduce_sum(t, group):
    """Sum t over the ranks in place (through host memory on a gloo group)."""
    if t.device.type == "cuda" and dist.get_backend(group) == "gloo":
        h = t.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


class ShardedImager:
    """This rank's share of one image, and the combined image.

    ``imager_factory(params, device)`` builds the per-rank imager (default:
    ``Imager``); it must offer reset, grid, image, stats, set_plane_range and
    set_weight_sum.
    """

    def __init__(self, params, device=None, group=None, mode="planes", imager_factory=None):
        from . import Imager, UNIFORM_WEIGHT
        if mode not in ("planes", "measurements"):
            raise ValueError("mode must be 'planes' or 'measurements'")
        if mode == "measurements" and int(params.get("flags", 0)) & UNIFORM_WEIGHT:
            raise ValueError("uniform weighting needs the density of every shard; use mode='planes'")
        self.mode = mode
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.imager = (imager_factory or Imager)(params, device)
        self.k0, self.k1 = (plane_share(int(params["nw"]), self.rank, self.world) if mode == "planes"
                            else (0, int(params["nw"])))
        self._range()

    def _range(self):
        if self.mode == "planes":
            self.imager.set_plane_range(self.k0, self.k1)

    def reset(self):
        self.imager.reset()
        self._range()

    def grid(self, vis, u, v, w, wt=None):
        """mode 'planes': all measurements; mode 'measurements': this rank's share."""
        self.imager.grid(vis, u, v, w, wt)

    def image(self, out=None):
        """The image of everything every rank gridded (on every rank)."""
        if self.mode == "measurements":
            sw = torch.tensor([float(self.imager.stats()["sum_weights"])], dtype=torch.float64)
            _all_reduce_sum(sw, self.group)
            self.imager.set_weight_sum(float(sw.item()))
        img = self.imager.image(out=out)
        return _all_reduce_sum(img, self.group)

    def close(self):
        self.imager.close()
