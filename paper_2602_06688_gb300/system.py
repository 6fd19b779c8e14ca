"""A multi-sensor adaptive-optics system through the C ABI.

Two ways to run one frame of every sensor, the concatenated slopes and the
reconstructor product (the multi-sensor systems of Sect. 6, Tab. 2):

* ``frame``: one persistent launch (specula_mwfs_frame) covering all
  sensors, their slopes and the MVM;
* ``frame_separate``: the single-sensor calls in sequence, one group of
  kernels per sensor (specula_atmo_extract, specula_sh_image /
  specula_pwfs_image, specula_slopes) and one specula_recon.

Both compute the same quantities; all arithmetic runs in libspecula_gb300 and
this class only owns buffers and issues the calls.
"""
import numpy as np

import synth
from . import (PREC_FP32, SLOPES_PYR, SLOPES_SH, Mwfs, ShDesc, layer_desc, pupil_desc,
               pwfs_desc, recon_desc, slopec_desc, source_desc, specula_atmo_extract,
               specula_graph_begin, specula_graph_end, specula_pupil_mask, specula_pwfs_image,
               specula_pwfs_plan, specula_recon, specula_screen_generate, specula_sh_image,
               specula_sh_plan, specula_slopes, specula_valid_subaps_host, wfs_desc)


class System:
    def __init__(self, ctx, wl, n_modes=None, R=None, seed_offset=0, with_separate=True,
                 device="cuda"):
        import torch
        self.torch, self.ctx, self.wl = torch, ctx, wl
        self.layers = [layer_desc(l) for l in wl.layers]
        self.screens = []
        for l in wl.layers:
            noise = torch.tensor(synth.screen_noise(l.seed + seed_offset, l.side), device=device)
            scr = torch.empty(l.side, l.side, device=device, dtype=torch.float32)
            specula_screen_generate(ctx, l.side, l.pitch_m, l.r0_m, l.L0_m, noise,
                                    synth.subharmonic_noise(l.seed + seed_offset), scr)
            del noise
            self.screens.append(scr)
        self.descs = [wfs_desc(s) for s in wl.sensors]
        # slope layout (the library's rule; checked against the plan below)
        self.n_valid = []
        for s in wl.sensors:
            nsub = s.pwfs.n_sub if s.kind == "pwfs" else s.sh.n_sub
            self.n_valid.append(len(specula_valid_subaps_host(pupil_desc(s.pupil), nsub)))
        self.offsets = list(np.cumsum([0] + [2 * v for v in self.n_valid])[:-1])
        self.n_slopes = int(sum(2 * v for v in self.n_valid))
        self.n_modes = n_modes if n_modes is not None else wl.n_modes
        if R is None and self.n_modes > 0:
            R = (synth.normal_draws(11 + seed_offset, (self.n_modes, self.n_slopes))
                 / np.sqrt(self.n_slopes)).astype(np.float32)
        self.R = None if R is None else torch.tensor(np.asarray(R, np.float32), device=device)
        self.m = Mwfs(ctx, self.descs, self.layers, self.screens, self.R)
        assert self.m.n_slopes == self.n_slopes and self.m.n_valid == self.n_valid
        self.slopes = torch.empty(self.n_slopes, device=device)
        self.ref = torch.empty(self.n_slopes, device=device)
        self.modes = torch.empty(max(self.n_modes, 1), device=device)
        self.m.reference(self.ref, self._modes_arg())
        self.t_dev = torch.zeros(1, dtype=torch.float64, device=device)
        self.graph = None
        if with_separate:
            self._setup_separate(device)
        torch.cuda.synchronize()

    def _modes_arg(self, modes=None):
        if self.n_modes == 0:
            return None
        return self.modes if modes is None else modes

    # ---- persistent launch ------------------------------------------------------
    def frame(self, t, t_dev=None, stream=None):
        self.m.frame(t, self.slopes, self._modes_arg(), ref=self.ref, t_dev=t_dev, stream=stream)
        return self.slopes, self.modes

    def capture(self, stream, separate=False):
        """One frame (persistent, or the per-sensor calls) as a CUDA graph
        reading the frame time from self.t_dev."""
        self.torch.cuda.synchronize()
        specula_graph_begin(self.ctx, stream)
        try:
            if separate:
                self.frame_separate(0.0, t_dev=self.t_dev, stream=stream)
            else:
                self.frame(0.0, t_dev=self.t_dev, stream=stream)
        finally:
            g = specula_graph_end(self.ctx, stream)
        return g

    # ---- single-sensor calls, one sensor after the other ------------------------
    def _setup_separate(self, device):
        torch, ctx = self.torch, self.ctx
        self.sep = []
        self.sep_slopes = torch.empty(self.n_slopes, device=device)
        self.sep_modes = torch.empty(max(self.n_modes, 1), device=device)
        self.sep_ref = torch.empty(self.n_slopes, device=device)
        for k, s in enumerate(self.wl.sensors):
            pu = pupil_desc(s.pupil)
            n = s.pupil.n_pix
            amp = torch.empty(n, n, device=device)
            specula_pupil_mask(ctx, pu, amp)
            valid = torch.tensor(specula_valid_subaps_host(pu, s.pwfs.n_sub if s.kind == "pwfs"
                                                           else s.sh.n_sub), device=device)
            e = {"pupil": pu, "src": source_desc(s.source), "amp": amp, "valid": valid,
                 "phase": torch.zeros(n, n, device=device), "kind": s.kind}
            if s.kind == "sh":
                g = s.sh
                e["sh"] = ShDesc(g.n_sub, g.sub_pix, g.fft_n)
                nv = specula_sh_plan(ctx, pu, e["sh"])
                assert nv == self.n_valid[k]
                e["img"] = torch.empty(nv, g.fft_n, g.fft_n, device=device)
                e["slopec"] = slopec_desc(SLOPES_SH, g.n_sub, valid, g.fft_n)
            else:
                e["pwfs"] = pwfs_desc(s.pwfs)
                specula_pwfs_plan(ctx, pu, e["pwfs"])
                e["img"] = torch.empty(2 * s.pwfs.n_sub, 2 * s.pwfs.n_sub, device=device)
                e["slopec"] = slopec_desc(SLOPES_PYR, s.pwfs.n_sub, valid)
            o = self.offsets[k]
            e["out"] = self.sep_slopes[o:o + 2 * self.n_valid[k]]
            e["ref"] = self.sep_ref[o:o + 2 * self.n_valid[k]]
            self.sep.append(e)
            # reference slopes: a flat wavefront
            self._image(e, None)
            specula_slopes(ctx, e["slopec"], e["img"], None, e["ref"])
        self.rec = (recon_desc(self.n_modes, self.n_slopes, PREC_FP32, self.R)
                    if self.R is not None else None)

    def _image(self, e, stream):
        ctx = self.ctx
        if e["kind"] == "sh":
            specula_sh_image(ctx, e["pupil"], e["sh"], e["amp"], e["phase"], e["img"],
                             e["img"].shape[0], stream=stream)
        else:
            specula_pwfs_image(ctx, e["pupil"], e["pwfs"], e["amp"], e["phase"], e["img"],
                               stream=stream)

    def frame_separate(self, t, t_dev=None, stream=None):
        ctx = self.ctx
        for e in self.sep:
            specula_atmo_extract(ctx, self.layers, self.screens, e["src"], e["pupil"], t,
                                 e["phase"], t_dev=t_dev, stream=stream)
            self._image(e, stream)
            specula_slopes(ctx, e["slopec"], e["img"], e["ref"], e["out"], stream=stream)
        if self.rec is not None:
            specula_recon(ctx, self.rec, self.sep_slopes, self.sep_modes, stream=stream)
        return self.sep_slopes, self.sep_modes
