"""Tile cache for the pyramid autotuner (specula_pwfs_autotune).

The library times candidate tilings on the device; this module remembers the
winner per (device name, pupil pixels, FFT side, modulation points, subaps,
batch) in a JSON file so later runs skip the search.  The cache location is
$SPECULA_TUNE_CACHE, else ~/.cache/specula_gb300/tiles.json.
"""
import json
import os

from . import specula_pwfs_autotune, specula_pwfs_set_tiles


def cache_path():
    return os.environ.get("SPECULA_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "specula_gb300", "tiles.json")


# bumped whenever the kernels' best tiling can change (v5: the two-pass form's
# column-major slot blocks and 128-thread row filter)
_VERSION = "v5"


def _key(device_name, pupil, pwfs, n_batch):
    return (f"{_VERSION}|{device_name}|np{pupil.n_pix}|pad{pwfs.pad}|mod{pwfs.n_mod}"
            f"|sub{pwfs.n_sub}|b{n_batch}")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass   # a read-only home only loses the cache, not the tuning


def tune_pwfs(ctx, pupil, pwfs, amp, phase, det, force=False, reps=3,
              max_workspace_bytes=512 << 20):
    """Apply the cached tiling for this geometry, or run the autotuner and
    cache its choice.  Returns (chunk, ka, passes, from_cache)."""
    import torch
    n = pupil.n_pix
    n_batch = phase.numel() // (n * n)
    key = _key(torch.cuda.get_device_name(ctx.device), pupil, pwfs, n_batch)
    d = _load()
    if not force and key in d:
        ch, ka, ps = d[key]
        specula_pwfs_set_tiles(ctx, pupil, pwfs, ch, ka, ps)
        return ch, ka, ps, True
    ch, ka, ps = specula_pwfs_autotune(ctx, pupil, pwfs, amp, phase, det, reps=reps,
                                       max_workspace_bytes=max_workspace_bytes)
    d[key] = [ch, ka, ps]
    _store(d)
    return ch, ka, ps, False
