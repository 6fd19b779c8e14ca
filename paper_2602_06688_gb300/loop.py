"""Closed adaptive-optics loop on one pyramid sensor: the atmosphere, a modal
deformable mirror subtracted from it, the pyramid frame (image, slopes,
calibrated modal reconstructor) and an integrator whose command reaches the
mirror one step later (the SOUL example's DM, IirFilter and ``:-1`` delayed
connection, App. B, Listing 2; Sect. 2.2).  Every step is a sequence of C-ABI
calls (graph-capturable); calibration uses the push-pull interaction matrix
and the float64 pseudo-inverse of the library.

Step k:
    residual = phi_atm(t_k) - B^T c_{k-1}
    m        = R (slopes(residual) - reference)
    c_k      = (1 - leak) c_{k-1} + gain m
with the residual's piston-free RMS and the Strehl ratio at the science
wavelength recorded per step in ``stats`` (two float64 on the device).
"""
from . import (PREC_FP32, recon_desc, specula_atmo_extract, specula_calib_intmat,
               specula_dm_shape, specula_graph_begin, specula_graph_end,
               specula_loop_integrate, specula_loop_residual, specula_modal_basis,
               specula_pinv_fp64, specula_pwfs_image, specula_recon, specula_slopes)
from .frame import PwfsFrame


class ClosedLoop:
    def __init__(self, ctx, wl, n_modes=None, gain=0.4, leak=0.01, push_amp=0.1, rcond=1e-3,
                 sci_wavelength_nm=1650.0, seed_offset=0, device="cuda"):
        import torch
        self.torch = torch
        self.ctx = ctx
        nm = n_modes or wl.n_modes
        # the frame supplies the atmosphere, the pupil, the pyramid plan, the
        # slope computer and its flat-wavefront reference
        self.fr = fr = PwfsFrame(ctx, wl, n_modes=nm, seed_offset=seed_offset, device=device)
        n = fr.n_pix
        self.n_modes = nm
        self.gain, self.leak = float(gain), float(leak)
        self.wfs_over_sci = fr.src.wavelength_nm / float(sci_wavelength_nm)
        # calibration: modal basis, push-pull interaction matrix, pseudo-inverse
        self.basis = torch.empty(nm, n, n, device=device)
        specula_modal_basis(ctx, fr.pupil, nm, self.basis)
        im = torch.empty(fr.n_slopes, nm, dtype=torch.float64, device=device)
        specula_calib_intmat(ctx, fr.pupil, fr.pwfs, fr.amp, self.basis, nm, push_amp, fr.slopec,
                             im)
        R64 = torch.empty(nm, fr.n_slopes, dtype=torch.float64, device=device)
        self.R = torch.empty(nm, fr.n_slopes, device=device)
        self.rank = specula_pinv_fp64(ctx, im, rcond, R64, self.R)
        del im, R64
        self.rec = recon_desc(nm, fr.n_slopes, PREC_FP32, self.R)
        self.cmd = torch.zeros(nm, device=device)
        self.dm = torch.zeros(n, n, device=device)
        self.resid = torch.zeros(n, n, device=device)
        self.stats = torch.zeros(2, dtype=torch.float64, device=device)
        self.graph = None
        self.t_dev = None
        torch.cuda.synchronize()

    def reset(self):
        self.cmd.zero_()

    def step(self, t, t_dev=None, stream=None):
        """Enqueue step k at time t (or *t_dev)."""
        ctx, fr = self.ctx, self.fr
        specula_atmo_extract(ctx, fr.layers, fr.screens, fr.src, fr.pupil, t, fr.phase,
                             t_dev=t_dev, stream=stream)
        specula_dm_shape(ctx, self.basis, self.cmd, self.dm, stream=stream)
        specula_loop_residual(ctx, fr.amp, fr.phase, self.dm, self.wfs_over_sci, self.resid,
                              self.stats, stream=stream)
        specula_pwfs_image(ctx, fr.pupil, fr.pwfs, fr.amp, self.resid, fr.det, stream=stream)
        specula_slopes(ctx, fr.slopec, fr.det, fr.ref, fr.slopes, stream=stream)
        specula_recon(ctx, self.rec, fr.slopes, fr.modes, stream=stream)
        specula_loop_integrate(ctx, self.gain, self.leak, fr.modes, self.cmd, stream=stream)
        return self.stats

    def capture(self, stream):
        """One step as a CUDA graph on `stream`, reading its time from t_dev."""
        torch = self.torch
        self.t_dev = torch.zeros(1, dtype=torch.float64, device=self.cmd.device)
        torch.cuda.synchronize()
        specula_graph_begin(self.ctx, stream)
        try:
            self.step(0.0, t_dev=self.t_dev, stream=stream)
        finally:
            self.graph = specula_graph_end(self.ctx, stream)
        return self.graph

    def replay(self, t, stream):
        with self.torch.cuda.stream(stream):
            self.t_dev.fill_(t)
        self.graph.launch(stream)
        return self.stats

    def close(self):
        if self.graph is not None:
            self.graph.close()
            self.graph = None
