"""One pyramid frame split across ranks by modulation point (the exchange is
one sum of detector images).

The modulated pyramid's image is a sum over modulation points, and binning is
linear.  Each rank therefore images the points of its own cosine slots
(``specula_pwfs_set_slots``), and one all-reduce of the detector gives every
rank the full image.  Slot c holds points c and n_mod - c; slots 0 and
n_mod / 2 hold one point each.  The ranges are contiguous slot blocks
balanced by point count.  Everything else in the frame (extraction, slopes,
reconstructor) runs on every rank; the detector is 147 KB at ELT scale.

This is the host side: it partitions and reduces.  The images are computed
by the library's kernels.
"""


def slot_points(n_mod, c):
    """The modulation points of cosine slot c."""
    return [c] if (c == 0 or 2 * c == n_mod) else [c, n_mod - c]


def slot_ranges(n_mod, world):
    """Contiguous [begin, end) slot blocks, one per rank: each block ends where
    the cumulative point count comes closest to the rank's share, so the
    counts differ by at most two (every slot holds one or two points).  Needs
    world <= n_mod // 2 + 1 (each rank at least one slot)."""
    nc = n_mod // 2 + 1
    if not 1 <= world <= nc:
        raise ValueError(f"{world} ranks for {nc} modulation slots")
    weights = [len(slot_points(n_mod, c)) for c in range(nc)]
    total = sum(weights)
    out, c = [], 0
    for r in range(world):
        begin = c
        target = total * (r + 1) / world
        done = sum(weights[:c])
        # take slots while that brings the cumulative count closer to the
        # target, leaving at least one slot for each remaining rank
        while c < nc - (world - r - 1) and (
                c == begin or abs(done + weights[c] - target) < abs(done - target)):
            done += weights[c]
            c += 1
        out.append((begin, c))
    out[-1] = (out[-1][0], nc)
    return out


class PointShardedImage:
    """The pyramid image of a frame on this rank's slots, then summed over the
    process group."""

    def __init__(self, ctx, pupil, pwfs, n_mod, group=None):
        import torch.distributed as dist
        from . import specula_pwfs_set_slots
        self.dist = dist
        self.group = group
        rank = dist.get_rank(group) if dist.is_initialized() else 0
        world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.ranges = slot_ranges(n_mod, world)
        self.begin, self.end = self.ranges[rank]
        self.ctx, self.pupil, self.pwfs = ctx, pupil, pwfs
        specula_pwfs_set_slots(ctx, pupil, pwfs, self.begin, self.end)

    def image(self, amp, phase, det, stream=None):
        """This rank's partial detector, then the sum over ranks in place."""
        from . import specula_pwfs_image
        specula_pwfs_image(self.ctx, self.pupil, self.pwfs, amp, phase, det, stream=stream)
        if self.dist.is_initialized() and self.dist.get_world_size(self.group) > 1:
            self.dist.all_reduce(det, group=self.group)
        return det
