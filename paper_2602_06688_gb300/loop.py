"""Closed adaptive-optics loop on one pyramid sensor: the atmosphere, a modal
deformable mirror subtracted from it, the pyramid frame (image, slopes,
calibrated modal reconstructor) and an integrator whose command reaches the
mirror one step later (the SOUL example's DM, IirFilter and ``:-1`` delayed
connection, App. B, Listing 2; Sect. 2.2).  Every step is a sequence of C-ABI
calls (graph-capturable); calibration uses the push-pull interaction matrix
and the float64 pseudo-inverse of the library.

Step k:
    residual = phi_atm(t_k) - B^T c_{k-1}
    m        = R s, with s = slopes(residual) - reference  (or a network's
               f(s), or R s + f(s): LoopNetwork)
    c_k      = (1 - leak) c_{k-1} + gain m
with the residual's piston-free RMS and the Strehl ratio at the science
wavelength recorded per step in ``stats`` (two float64 on the device).
"""
import numpy as np

import synth
from . import (PREC_FP32, recon_desc, specula_atmo_extract, specula_calib_intmat,
               specula_dm_shape, specula_graph_begin, specula_graph_end,
               specula_loop_integrate, specula_loop_residual, specula_modal_basis,
               specula_pinv_fp64, specula_pwfs_image, specula_recon, specula_slopes)
from .calibrated import noll_radial_orders
from .frame import PwfsFrame
from .learned import MlpRegressor


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
        # optional learned reconstructor in place of R (LoopNetwork)
        self.net = None
        self.xn = torch.empty(1, fr.n_slopes, device=device)
        self.dmodes = torch.empty(1, nm, device=device)
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
        net = self.net
        if net is None or net.residual:
            specula_recon(ctx, self.rec, fr.slopes, fr.modes, stream=stream)
        else:
            net.predict_into(fr.slopes.view(1, -1), fr.modes.view(1, -1), self.xn, stream=stream)
        specula_loop_integrate(ctx, self.gain, self.leak, fr.modes, self.cmd, stream=stream)
        if net is not None and net.residual:
            # m = R s + f(s): the correction enters the integrator with the
            # same gain (the leak is applied once, above)
            net.predict_into(fr.slopes.view(1, -1), self.dmodes, self.xn, stream=stream)
            specula_loop_integrate(ctx, self.gain, 0.0, self.dmodes.view(-1), self.cmd,
                                   stream=stream)
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


class LoopNetwork(MlpRegressor):
    """A learned reconstructor for the closed loop: slopes -> hidden ->
    hidden -> modes (GELU, the library's tcgen05 training kernels,
    weight-streaming inference at batch 1 inside the loop's graph), either
    in place of R (residual=False) or as a correction on top of it,
    m = R s + f(s) (residual=True: f learns what the linear reconstructor
    misses, the pyramid's non-linear response; R stays the fallback).

    Training pairs come from the regime the loop works in: synthetic modal
    phases B^T c, c ~ N(0, k sigma_n^2) per radial order n, sigma_n^2 the
    per-order mean square of the modes the loop reconstructs with R once
    settled (the closed-loop residual spectrum as the sensor sees it) and k
    (spectrum_scale) widening it to the larger residuals of the loop's
    transients; labels are the exact coefficients (minus R s for the
    correction).  Inputs and targets are scaled globally (each mode weighed
    by its variance, as the residual wavefront weighs it)."""

    def __init__(self, loop, hidden=(1024, 1024), residual=True):
        self.loop, self.ctx, self.torch = loop, loop.ctx, loop.torch
        self.n_slopes, self.n_modes, self.hidden = loop.fr.n_slopes, loop.n_modes, hidden
        self.residual = residual

    def residual_spectrum(self, steps=300, settle=100, t0=20.0):
        """Per-radial-order mean square of the reconstructed modes over a run
        of the loop with R (from a reset command, times t0 + k dt)."""
        torch, cl = self.torch, self.loop
        net, cl.net = cl.net, None
        cl.reset()
        acc = torch.zeros(self.n_modes, dtype=torch.float64, device="cuda")
        for k in range(steps):
            cl.step(t0 + k * cl.fr.dt)
            if k >= settle:
                acc += cl.fr.modes.view(-1).double() ** 2
        cl.net = net
        cl.reset()
        v = (acc / (steps - settle)).cpu().numpy()
        orders = noll_radial_orders(self.n_modes)
        return np.array([v[orders == n].mean() if np.any(orders == n) else 0.0
                         for n in range(orders.max() + 1)])

    def pairs(self, n_samples, seed, order_var, batch=256):
        """(slopes, coefficients) of phases B^T c through the loop's pyramid,
        slope computer and reference."""
        torch, cl = self.torch, self.loop
        fr = cl.fr
        n, nm = fr.n_pix, self.n_modes
        sig = np.sqrt(np.asarray(order_var, dtype=np.float64)[noll_radial_orders(nm)])
        sig_t = torch.tensor(sig.astype(np.float32), device="cuda")
        basis_t = cl.basis.reshape(nm, n * n).t().contiguous()
        synth_rec = recon_desc(n * n, nm, PREC_FP32, basis_t)
        X = torch.empty(n_samples, self.n_slopes, device="cuda")
        T = torch.empty(n_samples, nm, device="cuda")
        ph = torch.empty(batch, n, n, device="cuda")
        nd = fr.det.shape[-1]
        det = torch.empty(batch, nd, nd, device="cuda")
        for b0 in range(0, n_samples, batch):
            g = min(batch, n_samples - b0)
            c = torch.tensor(synth.normal_draws(seed * 1000003 + b0, (g, nm)).astype(np.float32),
                             device="cuda") * sig_t
            T[b0:b0 + g] = c
            specula_recon(self.ctx, synth_rec, c, ph[:g].reshape(g, n * n))
            specula_pwfs_image(self.ctx, fr.pupil, fr.pwfs, fr.amp, ph[:g], det[:g])
            specula_slopes(self.ctx, fr.slopec, det[:g], fr.ref, X[b0:b0 + g])
        torch.cuda.synchronize()
        return X, T

    def train(self, n_pairs=32768, epochs=30, lr=1e-3, lr_final=1e-5, spectrum_scale=16.0,
              seed=21):
        torch = self.torch
        order_var = self.residual_spectrum()
        X, T = self.pairs(n_pairs, seed, order_var * spectrum_scale)
        info = {"pairs": n_pairs, "epochs": epochs, "lr": [lr, lr_final],
                "spectrum_scale": spectrum_scale, "residual": self.residual}
        if self.residual:
            L = torch.empty_like(T)
            specula_recon(self.ctx, self.loop.rec, X, L)
            T = T - L
            info["linear_rel_err_on_pairs"] = float(T.norm() / (T + L).norm())
            del L
        hist = self.fit(X, T, epochs=epochs, lr=lr, lr_final=lr_final,
                        per_column_targets=False, per_column_inputs=False)
        info["final_loss"] = hist[-1]
        del X, T
        torch.cuda.synchronize()
        return info
