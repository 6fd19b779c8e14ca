"""Learned nonlinear reconstructor, trained on pairs the simulator generates.

Pipeline (every numerical step runs in libspecula_gb300 kernels):

1. training pairs: independent von Karman screens per sample (device Philox
   noise, specula_screen_generate_batch) scaled to a Fried parameter drawn
   uniformly per sample and cropped to the pupil (specula_random_phase,
   AtmoRandomPhase), imaged by the modulated pyramid, turned into slopes;
   labels are the true modal coefficients, the least-squares projection of
   each phase on the modal basis (ModalAnalysis) with the projector
   pinv(Z) computed in float64 on the GPU;
2. the linear baseline: push-pull interaction matrix and its truncated
   pseudo-inverse (ImCalibrator / RecCalibrator), applied as an MVM;
3. the network: slopes -> hidden -> hidden -> modes with GELU, inputs and
   outputs standardised per column, trained with Adam on the tcgen05 GEMMs;
4. evaluation on held-out samples: modal residual RMS of both reconstructors
   against the true coefficients.
"""
import math

import numpy as np

import synth
from . import (MLP, PREC_BF16X2, PREC_FP32, SLOPES_PYR, pupil_desc, pwfs_desc, recon_desc,
               slopec_desc, specula_affine_cols, specula_calib_intmat, specula_col_stats,
               specula_modal_basis, specula_modal_basis_host, specula_pinv_fp64,
               specula_pupil_mask, specula_pwfs_image, specula_pwfs_plan, specula_random_phase,
               specula_recon, specula_recon_convert, specula_screen_generate_batch,
               specula_slopes, specula_valid_subaps_host)


class MlpRegressor:
    """A slopes -> modes perceptron fitted on the device: inputs and outputs
    standardised per column, Kaiming-uniform start from a seed, Adam with a
    cosine learning-rate decay on the tcgen05 GEMMs.  Needs self.ctx,
    self.torch, self.n_slopes, self.n_modes and self.hidden."""

    def _stats(self, A):
        torch = self.torch
        m = torch.empty(A.shape[1], device="cuda")
        s = torch.empty(A.shape[1], device="cuda")
        specula_col_stats(self.ctx, A, m, s)
        torch.cuda.synchronize()
        mh, sh = m.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
        sh = np.where(sh > 1e-12, sh, 1.0)
        return mh, sh

    def fit(self, X, T, epochs=10, batch=256, lr=1e-3, lr_final=1e-4, init_seed=5,
            per_column_targets=True, per_column_inputs=True):
        """per_column_targets False scales every target column by the same
        factor (the largest column deviation), so the loss weighs each mode
        by its variance, as a residual-wavefront metric does, instead of
        equally; per_column_inputs False scales every input column by their
        RMS deviation, so inputs whose spectrum differs from the training
        set's are not magnified column by column."""
        torch = self.torch
        xm, xs = self._stats(X)
        tm, ts = self._stats(T)
        if not per_column_targets:
            ts = np.full_like(ts, ts.max())
        if not per_column_inputs:
            xs = np.full_like(xs, np.sqrt(np.mean(xs ** 2)))
        dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
        self.x_shift, self.x_mul = dev(xm), dev(1.0 / xs)
        self.t_shift, self.t_mul = dev(tm), dev(1.0 / ts)
        self.y_shift, self.y_mul = dev(-tm / ts), dev(ts)     # undo: y = yn * s + m
        Xn = torch.empty_like(X)
        Tn = torch.empty_like(T)
        specula_affine_cols(self.ctx, X, self.x_shift, self.x_mul, Xn)
        specula_affine_cols(self.ctx, T, self.t_shift, self.t_mul, Tn)
        sizes = (self.n_slopes, self.hidden[0], self.hidden[1], self.n_modes)
        self.mlp = MLP(self.ctx, sizes, max(batch, 1024))
        dims = list(sizes)
        for l in range(3):
            bound = 1.0 / math.sqrt(dims[l])
            W = synth.uniform_draws(init_seed * 100 + 2 * l, (dims[l + 1], dims[l]), -bound, bound)
            b = synth.uniform_draws(init_seed * 100 + 2 * l + 1, (dims[l + 1],), -bound, bound)
            self.mlp.set_layer(l, W, b)
        loss = torch.empty(1, device="cuda")
        n = X.shape[0]
        steps = max(1, epochs * (n // batch))
        hist, k = [], 0
        for ep in range(epochs):
            for b0 in range(0, n - batch + 1, batch):
                # cosine decay from lr to lr_final
                lr_k = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / steps))
                self.mlp.forward(Xn[b0:b0 + batch])
                self.mlp.backward(Tn[b0:b0 + batch], loss)
                self.mlp.adam(lr_k)
                k += 1
            hist.append(float(loss.item()))
        return hist

    def predict_into(self, X, Y, Xn, stream=None):
        """Y = network(X) into preallocated buffers (Xn: X's shape), every step
        a library call on `stream` (graph-capturable; batches of at most 4 take
        the weight-streaming inference kernels)."""
        specula_affine_cols(self.ctx, X, self.x_shift, self.x_mul, Xn, stream=stream)
        self.mlp.infer(Xn, Y, stream=stream)
        specula_affine_cols(self.ctx, Y, self.y_shift, self.y_mul, Y, stream=stream)

    def predict(self, X, chunk=1024):
        torch = self.torch
        Xn = torch.empty_like(X)
        specula_affine_cols(self.ctx, X, self.x_shift, self.x_mul, Xn)
        Y = torch.empty(X.shape[0], self.n_modes, device="cuda")
        for b0 in range(0, X.shape[0], chunk):
            b1 = min(X.shape[0], b0 + chunk)
            self.mlp.forward(Xn[b0:b1], Y[b0:b1])
        specula_affine_cols(self.ctx, Y, self.y_shift, self.y_mul, Y)
        return Y


class LearnedPipeline(MlpRegressor):
    def __init__(self, ctx, wl, n_modes=None, hidden=None, screen_side=256, push_amp=0.1,
                 rcond=1e-3, seed=77):
        import torch
        self.torch, self.ctx, self.wl = torch, ctx, wl
        s = wl.sensors[0]
        self.sensor = s
        self.pupil, self.pwfs = pupil_desc(s.pupil), pwfs_desc(s.pwfs)
        n = s.pupil.n_pix
        self.n = n
        self.n_modes = n_modes or wl.n_modes
        self.hidden = hidden or wl.mlp_hidden or (1024, 1024)
        self.side = screen_side
        self.seed = seed
        self.L0 = wl.layers[0].L0_m
        self.lam = s.source.wavelength_nm
        specula_pwfs_plan(ctx, self.pupil, self.pwfs)
        self.amp = torch.empty(n, n, device="cuda")
        specula_pupil_mask(ctx, self.pupil, self.amp)
        valid = specula_valid_subaps_host(self.pupil, s.pwfs.n_sub)
        self.idx = torch.tensor(valid, device="cuda")
        self.n_slopes = 2 * len(valid)
        self.slopec = slopec_desc(SLOPES_PYR, s.pwfs.n_sub, self.idx)
        nd = 2 * s.pwfs.n_sub
        self.nd = nd
        det = torch.empty(nd, nd, device="cuda")
        self.ref = torch.empty(self.n_slopes, device="cuda")
        specula_pwfs_image(ctx, self.pupil, self.pwfs, self.amp, torch.zeros(n, n, device="cuda"),
                           det)
        specula_slopes(ctx, self.slopec, det, None, self.ref)
        # modal basis and the float64 projector pinv(Z) over the full grid
        # (rows outside the pupil are zero, so they drop out of Z^T Z)
        self.basis = torch.empty(self.n_modes, n, n, device="cuda")
        specula_modal_basis(ctx, self.pupil, self.n_modes, self.basis)
        Zh = specula_modal_basis_host(self.pupil, self.n_modes).reshape(self.n_modes, n * n)
        Zf = torch.tensor(np.ascontiguousarray(Zh.T), device="cuda")        # (n^2, n_modes)
        P64 = torch.empty(self.n_modes, n * n, dtype=torch.float64, device="cuda")
        self.P = torch.empty(self.n_modes, n * n, device="cuda")
        self.proj_rank = specula_pinv_fp64(ctx, Zf, 1e-9, P64, self.P)
        del Zf, P64
        self.proj = recon_desc(self.n_modes, n * n, PREC_FP32, self.P)
        # linear baseline: push-pull IM and its truncated pseudo-inverse
        im = torch.empty(self.n_slopes, self.n_modes, dtype=torch.float64, device="cuda")
        specula_calib_intmat(ctx, self.pupil, self.pwfs, self.amp, self.basis, self.n_modes,
                             push_amp, self.slopec, im)
        R64 = torch.empty(self.n_modes, self.n_slopes, dtype=torch.float64, device="cuda")
        self.R = torch.empty(self.n_modes, self.n_slopes, device="cuda")
        self.rank = specula_pinv_fp64(ctx, im, rcond, R64, self.R)
        del im, R64
        self.rec = recon_desc(self.n_modes, self.n_slopes, PREC_FP32, self.R)
        # the same R as split bf16 (hi + lo): batches of 32 and more run it on
        # the tensor cores at float32-level error
        self.R_hi = torch.empty(self.R.shape, dtype=torch.int16, device="cuda")
        self.R_lo = torch.empty(self.R.shape, dtype=torch.int16, device="cuda")
        specula_recon_convert(ctx, self.R, PREC_BF16X2, self.R_hi, self.R_lo)
        self.rec_split = recon_desc(self.n_modes, self.n_slopes, PREC_BF16X2, self.R_hi,
                                    self.R_lo)
        torch.cuda.synchronize()

    # ------------------------------------------------------------------ data
    def make_pairs(self, n_samples, sample0, r0_range=(0.06, 0.20), batch=512):
        """(slopes (n, n_slopes), labels (n, n_modes)) on the device."""
        torch = self.torch
        n = self.n
        X = torch.empty(n_samples, self.n_slopes, device="cuda")
        T = torch.empty(n_samples, self.n_modes, device="cuda")
        r0 = synth.uniform_draws(self.seed * 1000003 + sample0, n_samples, *r0_range)
        # screens at r0 = 1 m scale as r0^(-5/6); radians at 500 nm -> at the WFS
        scale = torch.tensor((r0 ** (-5.0 / 6.0) * 500.0 / self.lam).astype(np.float32),
                             device="cuda")
        scr = torch.empty(batch, self.side, self.side, device="cuda")
        ph = torch.empty(batch, n, n, device="cuda")
        det = torch.empty(batch, self.nd, self.nd, device="cuda")
        for g0 in range(0, n_samples, batch):
            g = min(batch, n_samples - g0)
            specula_screen_generate_batch(self.ctx, g, self.side, self.pupil.pitch_m, 1.0, self.L0,
                                          self.seed, sample0 + g0, scr)
            specula_random_phase(self.ctx, scr, g, self.side, n, scale[g0:g0 + g], ph)
            specula_pwfs_image(self.ctx, self.pupil, self.pwfs, self.amp, ph[:g], det[:g])
            specula_slopes(self.ctx, self.slopec, det[:g], self.ref, X[g0:g0 + g])
            specula_recon(self.ctx, self.proj, ph[:g].reshape(g, n * n), T[g0:g0 + g])
        torch.cuda.synchronize()
        return X, T

    def linear(self, X, split_bf16=False):
        """Modes of the calibrated linear reconstructor: R in float32 (CUDA
        cores), or its split-bf16 copy (tensor cores from 32 frames on)."""
        Y = self.torch.empty(X.shape[0], self.n_modes, device="cuda")
        specula_recon(self.ctx, self.rec_split if split_bf16 else self.rec, X, Y)
        return Y

    def evaluate(self, X, T):
        """Modal residual RMS [rad] of both reconstructors and of the labels."""
        torch = self.torch
        ml = self.linear(X)
        ms = self.linear(X, split_bf16=True)
        mm = self.predict(X)
        torch.cuda.synchronize()
        t = T.cpu().numpy().astype(np.float64)
        res = {}
        for name, m in (("linear", ml), ("linear_split_bf16", ms), ("learned", mm)):
            d = m.cpu().numpy().astype(np.float64) - t
            res[name] = float(np.sqrt(np.mean(np.sum(d * d, axis=1))))
        res["labels"] = float(np.sqrt(np.mean(np.sum(t * t, axis=1))))
        return res
