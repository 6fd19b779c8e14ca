"""A pyramid-WFS frame through the C ABI: extraction -> image -> slopes -> MVM.

This is the per-time-step chain of the paper's SOUL example (App. B, Listing
2: atmo -> prop -> pyramid -> detector -> slopec -> rec), with the phase
screens generated on the device from seeded noise.  All arithmetic runs in
libspecula_gb300; this class only owns buffers and issues the calls.
"""
import numpy as np

import synth
from . import (PREC_BF16, PREC_BF16X2, PREC_FP32, SLOPES_PYR, SLOPES_PYR_MAPS, layer_desc,
               pupil_desc,
               pwfs_desc, recon_desc, slopec_desc, source_desc, specula_atmo_extract,
               specula_ccd, specula_loop_integrate, specula_pupil_mask, specula_pupil_mask_host,
               specula_pwfs_image,
               specula_pwfs_plan, specula_pyr_image_index_host, specula_recon,
               specula_recon_convert, specula_screen_generate, specula_slopes,
               specula_valid_subaps_host)


def seeded_reconstructor(n_modes, n_slopes, seed):
    """A seeded stand-in reconstructor (float32, N(0, 1/n_slopes)) for timing
    workloads whose calibration is not part of the measured frame."""
    return (synth.normal_draws(seed, (n_modes, n_slopes)) / np.sqrt(n_slopes)).astype(np.float32)


class PwfsFrame:
    def __init__(self, ctx, wl, sensor=0, precision=PREC_FP32, R=None, n_modes=None,
                 seed_offset=0, device="cuda", autotune=False, batch=1, noise=None,
                 infinite=None):
        """batch > 1: every step computes `batch` consecutive frames (times t,
        t + dt, ...) of the open-loop sequence together: one extraction per
        frame, then one pyramid call, one slope call and one MVM call over
        the whole batch.

        noise: None (noise-free detector) or a dict with ``photons`` (per frame
        over the pupil), ``qe``, ``ron`` (electrons RMS) and ``seed``: the
        detector image then carries photon and readout noise (the CCD call),
        frame index round(t / dt).

        infinite: None (periodic FFT screens of the workload's side) or a dict
        with ``side`` (ring side), ``n_st`` (stencil lines, default 2) and
        ``seed``: the layers then run on infinite screens, grown before each
        frame (batch 1 only)."""
        import torch
        self.torch = torch
        self.ctx = ctx
        s = wl.sensors[sensor]
        if s.kind != "pwfs":
            raise ValueError("sensor is not a pyramid")
        self.wl = wl
        self.pupil = pupil_desc(s.pupil)
        self.pwfs = pwfs_desc(s.pwfs)
        self.src = source_desc(s.source)
        self.layers = [layer_desc(l) for l in wl.layers]
        n = s.pupil.n_pix
        self.n_pix = n
        self.inf = None
        if infinite:
            if batch != 1:
                raise ValueError("infinite screens run one frame per step")
            from .infinite import InfiniteAtmosphere
            self.inf = InfiniteAtmosphere(ctx, wl.layers, s.source, s.pupil, infinite["side"],
                                          n_st=infinite.get("n_st", 2),
                                          seed=infinite.get("seed", 1), device=device)
            for d in self.layers:
                d.side = self.inf.side
        self.screens = [] if self.inf is None else self.inf.screens
        for l in (wl.layers if self.inf is None else ()):
            scr_noise = torch.tensor(synth.screen_noise(l.seed + seed_offset, l.side),
                                     device=device)
            scr = torch.empty(l.side, l.side, device=device, dtype=torch.float32)
            specula_screen_generate(ctx, l.side, l.pitch_m, l.r0_m, l.L0_m, scr_noise,
                                    synth.subharmonic_noise(l.seed + seed_offset), scr)
            del scr_noise
            self.screens.append(scr)
        self.amp = torch.empty(n, n, device=device)
        specula_pupil_mask(ctx, self.pupil, self.amp)
        # the quadrant layout when the four pupil images tile a pad-2 grid,
        # explicit image index maps for any other padding or separation
        self.quadrants = s.pwfs.pad == 2 and s.pwfs.pup_dist_px == n
        if self.quadrants:
            valid = specula_valid_subaps_host(self.pupil, s.pwfs.n_sub)
            self.valid = torch.tensor(valid, device=device)
            self.n_valid = len(valid)
        else:
            maps = specula_pyr_image_index_host(self.pupil, s.pwfs.pad, s.pwfs.pup_dist_px,
                                                s.pwfs.n_sub)
            self.valid = torch.tensor(maps.ravel(), device=device)
            self.n_valid = maps.shape[1]
        self.n_slopes = 2 * self.n_valid
        self.n_modes = n_modes or wl.n_modes
        specula_pwfs_plan(ctx, self.pupil, self.pwfs)
        d = s.pwfs.pad * s.pwfs.n_sub
        self.batch = batch
        self.dt = wl.dt_s
        if batch == 1:
            self.phase = torch.zeros(n, n, device=device)
            self.det = torch.empty(d, d, device=device)
            self.slopes = torch.empty(self.n_slopes, device=device)
            self.modes = torch.empty(self.n_modes, device=device)
        else:
            self.phase = torch.zeros(batch, n, n, device=device)
            self.det = torch.empty(batch, d, d, device=device)
            self.slopes = torch.empty(batch, self.n_slopes, device=device)
            self.modes = torch.empty(batch, self.n_modes, device=device)
        self.ref = torch.empty(self.n_slopes, device=device)
        self.noise = dict(noise) if noise else None
        self.frame_dev = torch.zeros(1, dtype=torch.int32, device=device)
        self.slopec = (slopec_desc(SLOPES_PYR, s.pwfs.n_sub, self.valid) if self.quadrants else
                       slopec_desc(SLOPES_PYR_MAPS, s.pwfs.pad * s.pwfs.n_sub, self.valid))
        if R is None:
            R = seeded_reconstructor(self.n_modes, self.n_slopes, seed=7 + seed_offset)
        self.R = torch.tensor(np.asarray(R, dtype=np.float32), device=device)
        self.learned = None
        self.learned_correction = False
        self.set_precision(precision)
        # reference slopes: a flat wavefront in the same geometry
        flat, fdet = torch.zeros(n, n, device=device), torch.empty(d, d, device=device)
        specula_pwfs_image(ctx, self.pupil, self.pwfs, self.amp, flat, fdet)
        specula_slopes(ctx, self.slopec, fdet, None, self.ref)
        if self.noise:
            # expected photo-electrons per unit of the image (it sums to the
            # number of pupil pixels)
            npup = float(specula_pupil_mask_host(self.pupil).sum())
            self.noise_scale = self.noise["photons"] * self.noise.get("qe", 1.0) / npup
        torch.cuda.synchronize()
        self.tiles = None
        if autotune:
            from .autotune import tune_pwfs
            for k in range(batch):
                specula_atmo_extract(ctx, self.layers, self.screens, self.src, self.pupil,
                                     k * self.dt, self.phase.view(batch, n, n)[k])
            self.tiles = tune_pwfs(ctx, self.pupil, self.pwfs, self.amp, self.phase, self.det,
                                   force=autotune == "force")
            torch.cuda.synchronize()

    def set_precision(self, precision):
        torch = self.torch
        self.precision = precision
        if precision == PREC_FP32:
            self.rec = recon_desc(self.n_modes, self.n_slopes, PREC_FP32, self.R)
            return
        self.R_hi = torch.empty(self.R.shape, dtype=torch.int16, device=self.R.device)
        self.R_lo = torch.empty(self.R.shape, dtype=torch.int16, device=self.R.device)
        specula_recon_convert(self.ctx, self.R, PREC_BF16X2, self.R_hi, self.R_lo)
        if precision == PREC_BF16:
            self.rec = recon_desc(self.n_modes, self.n_slopes, PREC_BF16, self.R_hi)
        elif precision == PREC_BF16X2:
            self.rec = recon_desc(self.n_modes, self.n_slopes, PREC_BF16X2, self.R_hi, self.R_lo)
        else:
            raise ValueError(precision)

    def capture(self, stream):
        """Record one frame into a CUDA graph on `stream` (a torch.cuda.Stream);
        the graph reads the frame time from self.t_dev."""
        from . import specula_graph_begin, specula_graph_end
        torch = self.torch
        self.t_dev = torch.zeros(self.batch, dtype=torch.float64, device=self.R.device)
        torch.cuda.synchronize()
        specula_graph_begin(self.ctx, stream)
        try:
            self.frame(0.0, t_dev=self.t_dev, stream=stream)
        finally:
            self.graph = specula_graph_end(self.ctx, stream)
        return self.graph

    def replay(self, t, stream):
        """Set the frame time and launch the captured frame on `stream`."""
        torch = self.torch
        if self.inf is not None:
            self.inf.advance(t, stream=stream)
        with torch.cuda.stream(stream):
            if self.noise:
                self.frame_dev.fill_(int(round(t / self.dt)))
            if self.batch == 1:
                self.t_dev.fill_(t)
            else:
                self.t_dev.copy_(t + self.dt * torch.arange(self.batch, dtype=torch.float64,
                                                            device=self.t_dev.device))
        self.graph.launch(stream)
        return self.modes

    def frame(self, t, t_dev=None, stream=None):
        """Enqueue one frame at time t (or *t_dev) on the current stream; with
        batch > 1 the frames at t, t + dt, ... (t_dev: one device time per
        frame)."""
        self.front(t, t_dev=t_dev, stream=stream)
        return self.reconstruct(stream=stream)

    def front(self, t, t_dev=None, stream=None, slopes=None):
        """The frame up to its slopes (extraction, image, detector noise,
        slopes) into `slopes` (default self.slopes)."""
        ctx = self.ctx
        slopes = self.slopes if slopes is None else slopes
        if self.inf is not None and t_dev is None:
            self.inf.advance(t, stream=stream)
        if self.batch == 1:
            specula_atmo_extract(ctx, self.layers, self.screens, self.src, self.pupil, t,
                                 self.phase, t_dev=t_dev, stream=stream)
        else:
            n = self.n_pix
            for k in range(self.batch):
                specula_atmo_extract(ctx, self.layers, self.screens, self.src, self.pupil,
                                     t + k * self.dt, self.phase.view(self.batch, n, n)[k],
                                     t_dev=None if t_dev is None else t_dev[k:k + 1],
                                     stream=stream)
        specula_pwfs_image(ctx, self.pupil, self.pwfs, self.amp, self.phase, self.det,
                           stream=stream)
        if self.noise:
            # eager: frame index from t; captured: from self.frame_dev
            k = 0 if t_dev is not None else int(round(t / self.dt))
            specula_ccd(ctx, self.det, self.noise_scale, self.noise.get("ron", 0.0),
                        self.noise.get("seed", 1), k, self.det,
                        frame_dev=self.frame_dev if t_dev is not None else None, stream=stream)
        specula_slopes(ctx, self.slopec, self.det, self.ref, slopes, stream=stream)
        return slopes

    def reconstruct(self, slopes=None, modes=None, stream=None):
        """Modes of `slopes` (default self.slopes) into `modes` (default
        self.modes): the MVM, the network in its place, or R s + f(s)."""
        ctx = self.ctx
        slopes = self.slopes if slopes is None else slopes
        modes = self.modes if modes is None else modes
        if self.learned is not None and not self.learned_correction:
            self.learned.infer(slopes.view(self.batch, -1), modes.view(self.batch, -1),
                               stream=stream)
        else:
            specula_recon(ctx, self.rec, slopes, modes, stream=stream)
            if self.learned is not None:
                # m = R s + f(s): the network's correction added by the
                # library's integrator update (gain 1, no leak: an exact sum)
                self.learned.infer(slopes.view(self.batch, -1), self.dmodes, stream=stream)
                specula_loop_integrate(ctx, 1.0, 0.0, self.dmodes.view(-1), modes.view(-1),
                                       stream=stream)
        return modes

    def use_learned(self, mlp, correction=False):
        """Reconstruct with a learned network (an MLP handle sized n_slopes ->
        ... -> n_modes) instead of the linear MVM, or with correction=True as
        a correction on top of it (m = R s + f(s)); None restores the MVM."""
        self.learned = mlp
        self.learned_correction = bool(correction) and mlp is not None
        if self.learned_correction:
            self.dmodes = self.torch.empty(self.batch, self.n_modes, device=self.modes.device)
