"""Partitions of the sensing chain across ranks, each with one exchange step
(the object placement across processes of Sect. 5 and the DistributedSH of
Sect. 6, App. A Tab. 4):

* one pyramid frame by modulation point: each rank images its cosine
  slots, one all-reduce of the detector (``PointShardedImage``);
* one Shack-Hartmann sensor by blocks of valid subapertures: each rank
  images its block and computes its slopes, one all-gather of slopes
  (``SubapShardedSH``);
* a multi-sensor system by sensor: each rank runs the chains of its
  sensors, one all-gather of the slope vectors (``SensorShards``);
* the reconstructor by mode rows: each rank multiplies its rows of R with
  the full slope vector, one all-gather of modes (``ModeRowRecon``).

Remote data is copied into local memory by the collective; nothing reads
another GPU's memory directly.  The modulation-point partition:

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


def block_ranges(n, world):
    """Contiguous [begin, end) blocks of n items, one per rank, sizes
    differing by at most one (the first n % world blocks one longer)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(n, world)
    out, b = [], 0
    for k in range(world):
        e = b + q + (1 if k < r else 0)
        out.append((b, e))
        b = e
    return out


def balanced_assignment(costs, world):
    """Sensors to ranks: greedy on decreasing cost (ties by index), each
    sensor to the least-loaded rank (lowest rank on ties).  Returns one sorted
    index list per rank."""
    load = [0.0] * world
    owner = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        owner[r].append(i)
    return [sorted(o) for o in owner]


def _all_gather_var(dist, group, piece, sizes):
    """All-gather of 1-D pieces of the given sizes (padded to the largest);
    returns the pieces in rank order."""
    import torch
    width = max(max(sizes), 1)
    buf = torch.zeros(width, dtype=piece.dtype, device=piece.device)
    buf[:piece.numel()] = piece.reshape(-1)
    bufs = [torch.empty_like(buf) for _ in sizes]
    dist.all_gather(bufs, buf, group=group)
    return [b[:n] for b, n in zip(bufs, sizes)]


def join_xy(pieces):
    """Full slope vector (all x then all y) from per-block vectors, each all
    x then all y of its block."""
    import torch
    xs = [p[:p.numel() // 2] for p in pieces]
    ys = [p[p.numel() // 2:] for p in pieces]
    return torch.cat(xs + ys)


class SubapShardedSH:
    """One Shack-Hartmann sensor split across ranks by contiguous blocks of
    its valid subapertures: every rank images its block
    (``specula_sh_set_range``) and computes its centre-of-gravity slopes, and
    one all-gather of slopes assembles the sensor's full vector on every
    rank."""

    def __init__(self, ctx, pupil, sh, n_valid, group=None, device="cuda"):
        import torch
        import torch.distributed as dist
        from . import SLOPES_SH, slopec_desc, specula_sh_set_range
        self.dist, self.group, self.torch = dist, group, torch
        init = dist.is_initialized()
        self.rank = dist.get_rank(group) if init else 0
        self.world = dist.get_world_size(group) if init else 1
        self.ranges = block_ranges(n_valid, self.world)
        self.begin, self.end = self.ranges[self.rank]
        self.count = self.end - self.begin
        self.ctx, self.pupil, self.sh = ctx, pupil, sh
        specula_sh_set_range(ctx, pupil, sh, self.begin, self.end)
        self.spots = torch.empty(self.count, sh.fft_n, sh.fft_n, device=device)
        idx = torch.zeros(max(self.count, 1), dtype=torch.int32, device=device)
        self.slopec = slopec_desc(SLOPES_SH, sh.n_sub, idx, sh.fft_n)
        self.slopec.n_valid = self.count
        self.part = torch.empty(2 * self.count, device=device)

    def slopes(self, amp, phase, ref=None, stream=None):
        """This rank's block of slopes, then the full vector (all x, all y)."""
        from . import specula_sh_image, specula_slopes
        specula_sh_image(self.ctx, self.pupil, self.sh, amp, phase, self.spots, self.count,
                         stream=stream)
        r = None
        if ref is not None:
            b, e, n = self.begin, self.end, ref.numel() // 2
            r = self.torch.cat([ref[b:e], ref[n + b:n + e]])
        specula_slopes(self.ctx, self.slopec, self.spots, r, self.part, stream=stream)
        if self.world == 1:
            return self.part.clone()
        pieces = _all_gather_var(self.dist, self.group, self.part,
                                 [2 * (e - b) for b, e in self.ranges])
        return join_xy(pieces)


class SensorShards:
    """A multi-sensor system split across ranks by sensor.  ``mine`` lists
    this rank's sensors (balanced by cost); after each rank has computed the
    slope vectors of its sensors, ``join`` all-gathers them and returns the
    system's vector in sensor order (each sensor all x then all y)."""

    def __init__(self, costs, sizes, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        init = dist.is_initialized()
        self.rank = dist.get_rank(group) if init else 0
        self.world = dist.get_world_size(group) if init else 1
        self.sizes = list(sizes)
        self.owners = balanced_assignment(costs, self.world)
        self.mine = self.owners[self.rank]

    def join(self, my_slopes):
        """my_slopes: {sensor index: its slope vector} for this rank's sensors."""
        import torch
        local = torch.cat([my_slopes[i].reshape(-1) for i in self.mine]) if self.mine else \
            torch.zeros(0, device=next(iter(my_slopes.values())).device if my_slopes else "cpu")
        if self.world == 1:
            return local
        sizes = [sum(self.sizes[i] for i in o) for o in self.owners]
        pieces = _all_gather_var(self.dist, self.group, local, sizes)
        per = {}
        for o, piece in zip(self.owners, pieces):
            off = 0
            for i in o:
                per[i] = piece[off:off + self.sizes[i]]
                off += self.sizes[i]
        return torch.cat([per[i] for i in range(len(self.sizes))])


class ModeRowRecon:
    """The modal reconstructor m = R s split across ranks by mode rows: every
    rank multiplies its contiguous block of R's rows with the full slope
    vector (``specula_recon`` on a row block, no copy of R), and one
    all-gather of modes gives every rank the full vector."""

    def __init__(self, ctx, R, group=None):
        import torch.distributed as dist
        from . import PREC_FP32, recon_desc
        self.dist, self.group = dist, group
        init = dist.is_initialized()
        self.rank = dist.get_rank(group) if init else 0
        self.world = dist.get_world_size(group) if init else 1
        n_modes, n_slopes = R.shape
        self.ranges = block_ranges(n_modes, self.world)
        b, e = self.ranges[self.rank]
        self.rows = R[b:e]
        self.desc = recon_desc(e - b, n_slopes, PREC_FP32, self.rows)
        self.ctx = ctx
        self.part = R.new_empty(e - b)

    def modes(self, slopes, stream=None):
        from . import specula_recon
        if self.part.numel():
            specula_recon(self.ctx, self.desc, slopes, self.part, stream=stream)
        if self.world == 1:
            return self.part.clone()
        import torch
        return torch.cat(_all_gather_var(self.dist, self.group, self.part,
                                         [e - b for b, e in self.ranges]))
