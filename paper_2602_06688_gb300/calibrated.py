"""The ELT pyramid's calibrated reconstructors compared at equal wavefront
accuracy: float32, split bf16 and bf16 MVMs of one calibrated R, and a
learned network (alone, or as a correction on top of R), by the residual
wavefront they leave.

Calibration (ImCalibrator / RecCalibrator, App. A, Tab. 4) on the device:
the Zernike modal basis (Kintner's recurrence), the push-pull interaction
matrix and its float64 truncated pseudo-inverse.  Accuracy metric: for a
phase phi and reconstructed modes m, the residual r = phi - B^T m over the
pupil (the mirror's correction, specula_dm_shape) and its piston-free RMS
(specula_loop_residual), averaged over held-out phases; no projector onto
the basis is needed.  Held-out phases: the ELT system's own 35-layer
atmosphere at frame times not used elsewhere, scaled to a closed-loop-like
RMS (the pyramid's linear range).  The network learns on synthetic modal
phases phi = B^T c with c drawn per radial order n with variance
proportional to (n + 1)^(-11/3) (the Kolmogorov Zernike spectrum), so its
labels are exact.  Every numerical step runs in libspecula_gb300 kernels.
"""
import numpy as np

import synth
from . import (PREC_BF16, PREC_BF16X2, PREC_FP32, recon_desc, specula_atmo_extract,
               specula_calib_intmat, specula_dm_shape, specula_loop_residual,
               specula_modal_basis, specula_pinv_fp64, specula_pwfs_image, specula_recon,
               specula_recon_convert, specula_slopes)
from .learned import MlpRegressor


def noll_radial_orders(n_modes):
    """Radial order n of the Noll modes j = 2 .. n_modes + 1."""
    out = np.empty(n_modes, dtype=np.int64)
    n, j = 1, 2
    for q in range(n_modes):
        while (n + 1) * (n + 2) // 2 < j:
            n += 1
        out[q] = n
        j += 1
    return out


class CalibratedRecon(MlpRegressor):
    def __init__(self, ctx, frame, n_modes=4000, push_amp=0.1, rcond=3e-2,
                 hidden=(2048, 2048)):
        import torch
        self.torch, self.ctx, self.fr = torch, ctx, frame
        fr = frame
        self.n, self.n_modes, self.n_slopes = fr.n_pix, n_modes, fr.n_slopes
        self.hidden = hidden
        n = self.n
        self.basis = torch.empty(n_modes, n, n, device="cuda")
        specula_modal_basis(ctx, fr.pupil, n_modes, self.basis)
        im = torch.empty(fr.n_slopes, n_modes, dtype=torch.float64, device="cuda")
        specula_calib_intmat(ctx, fr.pupil, fr.pwfs, fr.amp, self.basis, n_modes, push_amp,
                             fr.slopec, im)
        R64 = torch.empty(n_modes, fr.n_slopes, dtype=torch.float64, device="cuda")
        self.R = torch.empty(n_modes, fr.n_slopes, device="cuda")
        self.rank = specula_pinv_fp64(ctx, im, rcond, R64, self.R)
        del im, R64
        self.R_hi = torch.empty(self.R.shape, dtype=torch.int16, device="cuda")
        self.R_lo = torch.empty(self.R.shape, dtype=torch.int16, device="cuda")
        specula_recon_convert(ctx, self.R, PREC_BF16X2, self.R_hi, self.R_lo)
        self.recs = {
            "fp32": recon_desc(n_modes, fr.n_slopes, PREC_FP32, self.R),
            "bf16x2": recon_desc(n_modes, fr.n_slopes, PREC_BF16X2, self.R_hi, self.R_lo),
            "bf16": recon_desc(n_modes, fr.n_slopes, PREC_BF16, self.R_hi)}
        self.dm = torch.empty(n, n, device="cuda")
        self.res = torch.empty(n, n, device="cuda")
        self.stats = torch.zeros(2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()

    # ------------------------------------------------------------------ metric
    def residual_rms(self, phases, modes):
        """Mean over samples of the piston-free RMS [rad at the WFS] of
        phi - B^T m over the pupil."""
        torch = self.torch
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        for k in range(phases.shape[0]):
            specula_dm_shape(self.ctx, self.basis, modes[k], self.dm)
            specula_loop_residual(self.ctx, self.fr.amp, phases[k], self.dm, 1.0, self.res,
                                  self.stats)
            acc += self.stats[0]
        return float(acc.item()) / phases.shape[0]

    def slopes_of(self, phases, batch=32):
        """Reference-subtracted pyramid slopes of a stack of phases."""
        torch = self.torch
        fr = self.fr
        nb = phases.shape[0]
        X = torch.empty(nb, self.n_slopes, device="cuda")
        nd = fr.det.shape[-1]
        det = torch.empty(batch, nd, nd, device="cuda")
        for b0 in range(0, nb, batch):
            g = min(batch, nb - b0)
            specula_pwfs_image(self.ctx, fr.pupil, fr.pwfs, fr.amp, phases[b0:b0 + g], det[:g])
            specula_slopes(self.ctx, fr.slopec, det[:g], fr.ref, X[b0:b0 + g])
        return X

    # ------------------------------------------------------------------ data
    def heldout_phases(self, n_frames, t0, rms):
        """The system's atmosphere at frames t0, t0 + dt, ... scaled so the
        pupil RMS of each phase is `rms` rad (closed-loop-like residuals)."""
        torch = self.torch
        fr = self.fr
        n = self.n
        out = torch.empty(n_frames, n, n, device="cuda")
        inside = fr.amp > 0
        for k in range(n_frames):
            specula_atmo_extract(self.ctx, fr.layers, fr.screens, fr.src, fr.pupil,
                                 t0 + k * fr.dt, out[k])
            ph = out[k]
            v = ph[inside]
            ph.sub_(v.mean()).mul_(rms / float(v.std()))
            ph.mul_(fr.amp)
        return out

    def modal_pairs(self, n_samples, seed, rms, batch=256, order_var=None):
        """(slopes, coefficients) of synthetic modal phases B^T c, c ~ N(0,
        sigma_n^2): sigma_n^2 per radial order n from order_var (indexed by
        n), else (n + 1)^(-11/3); scaled to `rms` rad."""
        torch = self.torch
        n, nm = self.n, self.n_modes
        orders = noll_radial_orders(nm)
        if order_var is None:
            sig = (orders + 1.0) ** (-11.0 / 6.0)
        else:
            sig = np.sqrt(np.asarray(order_var, dtype=np.float64)[orders])
        sig *= rms / np.sqrt(np.sum(sig ** 2))            # expected RMS over the disk
        sig_t = torch.tensor(sig.astype(np.float32), device="cuda")
        if not hasattr(self, "basis_t"):
            self.basis_t = self.basis.reshape(nm, n * n).t().contiguous()   # (n^2, n_modes)
            self.synth_rec = recon_desc(n * n, nm, PREC_FP32, self.basis_t)
        X = torch.empty(n_samples, self.n_slopes, device="cuda")
        T = torch.empty(n_samples, nm, device="cuda")
        ph = torch.empty(batch, n, n, device="cuda")
        for b0 in range(0, n_samples, batch):
            g = min(batch, n_samples - b0)
            c = torch.tensor(synth.normal_draws(seed * 1000003 + b0, (g, nm)).astype(np.float32),
                             device="cuda") * sig_t
            T[b0:b0 + g] = c
            specula_recon(self.ctx, self.synth_rec, c, ph[:g].reshape(g, n * n))
            X[b0:b0 + g] = self.slopes_of(ph[:g])
        torch.cuda.synchronize()
        return X, T

    # ------------------------------------------------------------------ study
    def compare(self, n_test=64, n_train=32768, rms=0.3, epochs=40, t0=10.0, lr=1e-4,
                lr_final=1e-6):
        """Residual RMS of every reconstructor on the same held-out phases."""
        torch = self.torch
        phases = self.heldout_phases(n_test, t0, rms)
        X = self.slopes_of(phases)
        out = {"n_test": n_test, "phase_rms_rad": rms, "rank": self.rank,
               "no_correction": self.residual_rms(phases, torch.zeros(n_test, self.n_modes,
                                                                      device="cuda"))}
        for name, rec in self.recs.items():
            m = torch.empty(n_test, self.n_modes, device="cuda")
            specula_recon(self.ctx, rec, X, m)
            out[name] = self.residual_rms(phases, m)
        # the training spectrum: the per-radial-order variance of the linear
        # reconstruction of other frames of the same atmosphere
        tr = self.heldout_phases(64, t0 + 100.0, rms)
        mt = torch.empty(64, self.n_modes, device="cuda")
        specula_recon(self.ctx, self.recs["fp32"], self.slopes_of(tr), mt)
        v = (mt * mt).mean(dim=0).double().cpu().numpy()
        orders = noll_radial_orders(self.n_modes)
        order_var = np.array([v[orders == k].mean() if np.any(orders == k) else 0.0
                              for k in range(orders.max() + 1)])
        del tr, mt
        Xt, Tt = self.modal_pairs(n_train, 11, rms, order_var=order_var)
        # Adam steps of 1e-3 on the 13344-wide first layer move every unit's
        # pre-activation by O(10) within a few steps and the GELUs saturate;
        # 1e-4 trains
        hist = self.fit(Xt, Tt, epochs=epochs, lr=lr, lr_final=lr_final,
                        per_column_targets=False, per_column_inputs=False)
        out["learned"] = self.residual_rms(phases, self.predict(X))
        out["learned_train"] = {"pairs": n_train, "epochs": epochs, "lr": [lr, lr_final],
                                "final_loss": hist[-1]}
        # the network as a correction on top of R: m = R s + f(s), f trained on
        # what the float32 R misses on the same pairs
        Lt = torch.empty_like(Tt)
        specula_recon(self.ctx, self.recs["fp32"], Xt, Lt)
        hist_c = self.fit(Xt, Tt - Lt, epochs=epochs, lr=lr, lr_final=lr_final,
                          per_column_targets=False, per_column_inputs=False)
        del Xt, Tt, Lt
        m_lin = torch.empty(n_test, self.n_modes, device="cuda")
        specula_recon(self.ctx, self.recs["fp32"], X, m_lin)
        out["learned_correction"] = self.residual_rms(phases, m_lin + self.predict(X))
        out["learned_train"]["correction_final_loss"] = hist_c[-1]
        torch.cuda.synchronize()
        return out
