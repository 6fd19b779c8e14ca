"""Python binding of libspecula_gb300 (GB300-native wavefront-sensor hot path).

Each function has the name of the C entry point it wraps
(include/specula_gb300.h) and only marshals arguments: torch tensors supply
device memory (``data_ptr``) and the current CUDA stream; every computation
runs in the library's CUDA kernels.  A missing library raises ImportError at
first use — there is no fallback path.
"""
import ctypes as C
import weakref

import numpy as np

from . import _abi
from ._abi import (  # noqa: F401
    PupilDesc, SourceDesc, LayerDesc, PwfsDesc, ShDesc, SlopecDesc, ReconDesc, WfsDesc, InfLine,
    InfMove, INF_MAX_TASKS,
    SpeculaError, SLOPES_PYR, SLOPES_SH, SLOPES_PYR_MAPS, PWFS_FORM_TILT, PWFS_FORM_SHIFTED,
    PWFS_FORM_DFTGEMM_BF16, PWFS_FORM_DFTGEMM_TF32, PREC_FP32, PREC_BF16,
    PREC_BF16X2,
    OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ENONFINITE, ENOPLAN,
)


def lib():
    return _abi.load()


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor, after shape/dtype checks."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return C.c_void_p(t.data_ptr())


# ---- descriptor helpers (from the synth workload records) --------------------

def pupil_desc(p):
    return PupilDesc(int(p.n_pix), float(p.pitch_m), float(p.obsc_frac))


def source_desc(s):
    return SourceDesc(float(s.theta_x_rad), float(s.theta_y_rad), float(s.height_m),
                      float(s.wavelength_nm))


def layer_desc(l):
    return LayerDesc(int(l.side), float(l.pitch_m), float(l.height_m), float(l.vx_mps),
                     float(l.vy_mps))


def pwfs_desc(g):
    return PwfsDesc(int(g.pad), int(g.n_mod), int(g.n_sub), int(g.pup_dist_px),
                    float(g.mod_amp))


def sh_desc(g):
    return ShDesc(int(g.n_sub), int(g.sub_pix), int(g.fft_n))


# ---- context ------------------------------------------------------------------

class Context:
    """Owns a specula_ctx handle (plans, tables, device status word)."""

    def __init__(self, device=0):
        h = C.c_void_p()
        _abi.check(lib().specula_ctx_create(C.byref(h), int(device)), "specula_ctx_create")
        self.handle = h
        self.device = device
        # models created on this context; closed first so none outlives it
        self._children = weakref.WeakSet()

    def close(self):
        if self.handle:
            for ch in list(self._children):
                ch.close()
            lib().specula_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def _as_parameter_(self):
        return self.handle


def specula_last_cuda_error():
    """Text of the CUDA error behind this thread's last SPECULA_ECUDA."""
    return lib().specula_last_cuda_error().decode()


def specula_ctx_create(device=0):
    return Context(device)


def specula_ctx_destroy(ctx):
    ctx.close()


def specula_ctx_status(ctx):
    v = C.c_int32()
    _abi.check(lib().specula_ctx_status(ctx.handle, C.byref(v)), "specula_ctx_status")
    return v.value


def specula_ctx_set_guard(ctx, on):
    _abi.check(lib().specula_ctx_set_guard(ctx.handle, int(on)), "specula_ctx_set_guard")


def specula_check_guards(ctx):
    """(buffers compared, buffers whose guard band past the end changed)."""
    nc, nb = C.c_int32(), C.c_int32()
    _abi.check(lib().specula_check_guards(ctx.handle, C.byref(nc), C.byref(nb)),
               "specula_check_guards")
    return nc.value, nb.value


(K_PWFS_ROWS_FWD, K_PWFS_COLS, K_PWFS_ROWS_INV, K_ATMO, K_SLOPES, K_RECON, K_SH,
 K_PWFS_FIELD, K_PWFS_BIN, K_CALIB, K_GEMM, K_MLP, K_MWFS, K_PWFS_ROWFILT,
 K_PWFS_COLFILT, K_PWFS_SM_FWD, K_PWFS_SM_ROWS, K_PWFS_SM_COLS, K_LOOP, K_CCD,
 K_INFSCREEN, K_PEAK, K_PWFS_DFTGEMM) = range(23)
K_COUNT = 23
KERNEL_NAMES = ["pwfs_rows_fwd", "pwfs_cols", "pwfs_rows_inv", "atmo_extract", "slopes",
                "recon", "sh_spots", "pwfs_field", "pwfs_bin", "calib", "gemm", "mlp", "mwfs",
                "pwfs_rowfilt", "pwfs_colfilt_bin", "pwfs_sm_fwd", "pwfs_sm_rows",
                "pwfs_sm_colfilt_bin", "loop", "ccd", "infscreen", "fma_probe", "pwfs_dftgemm"]


def specula_prof_enable(ctx, capacity):
    _abi.check(lib().specula_prof_enable(ctx.handle, int(capacity)), "specula_prof_enable")


def specula_prof_read(ctx):
    """Returns {kernel name: (total ms, records)} since the last read."""
    ms = np.zeros(K_COUNT, dtype=np.float64)
    n = np.zeros(K_COUNT, dtype=np.int64)
    _abi.check(lib().specula_prof_read(ctx.handle, ms.ctypes.data_as(C.c_void_p),
                                       n.ctypes.data_as(C.c_void_p)), "specula_prof_read")
    return {KERNEL_NAMES[k]: (float(ms[k]), int(n[k])) for k in range(K_COUNT) if n[k]}


def specula_launch_count(ctx):
    v = C.c_int64()
    _abi.check(lib().specula_launch_count(ctx.handle, C.byref(v)), "specula_launch_count")
    return v.value


class Graph:
    """An instantiated CUDA graph of per-frame calls (specula_graph_*)."""

    def __init__(self, handle):
        self.handle = handle

    def launch(self, stream=None):
        _abi.check(lib().specula_graph_launch(self.handle, _stream(stream)),
                   "specula_graph_launch")

    def kernel_count(self):
        v = C.c_int64()
        _abi.check(lib().specula_graph_kernel_count(self.handle, C.byref(v)),
                   "specula_graph_kernel_count")
        return v.value

    def close(self):
        if self.handle:
            lib().specula_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def specula_graph_begin(ctx, stream):
    _abi.check(lib().specula_graph_begin(ctx.handle, _stream(stream)), "specula_graph_begin")


def specula_graph_end(ctx, stream):
    h = C.c_void_p()
    _abi.check(lib().specula_graph_end(ctx.handle, _stream(stream), C.byref(h)),
               "specula_graph_end")
    return Graph(h)


def specula_graph_launch(graph, stream=None):
    graph.launch(stream)


def specula_graph_kernel_count(graph):
    return graph.kernel_count()


def specula_graph_destroy(graph):
    graph.close()


def specula_strerror(status):
    return lib().specula_strerror(int(status)).decode()


def specula_version():
    return lib().specula_version()


# ---- integer geometry ------------------------------------------------------------

def specula_pupil_mask_host(pupil):
    n = pupil.n_pix
    out = np.zeros((n, n), dtype=np.uint8)
    _abi.check(lib().specula_pupil_mask_host(C.byref(pupil), out.ctypes.data_as(C.c_void_p)),
               "specula_pupil_mask_host")
    return out


def specula_valid_subaps_host(pupil, n_sub):
    idx = np.zeros(n_sub * n_sub, dtype=np.int32)
    nv = C.c_int32()
    _abi.check(lib().specula_valid_subaps_host(C.byref(pupil), int(n_sub),
                                               idx.ctypes.data_as(C.c_void_p), C.byref(nv)),
               "specula_valid_subaps_host")
    return idx[:nv.value].copy()


def specula_pyr_image_index_host(pupil, pad, pup_dist_px, n_sub):
    """(4, n_valid) int32 detector indices of the four pupil images of each
    valid subaperture (Q1..Q4) on the pad n_sub detector."""
    buf = np.zeros(4 * n_sub * n_sub, dtype=np.int32)
    nv = C.c_int32()
    _abi.check(lib().specula_pyr_image_index_host(C.byref(pupil), int(pad), int(pup_dist_px),
                                                  int(n_sub), buf.ctypes.data_as(C.c_void_p),
                                                  C.byref(nv)), "specula_pyr_image_index_host")
    return buf[:4 * nv.value].reshape(4, nv.value).copy()


def specula_mod_table_host(n_mod):
    c = np.zeros(n_mod)
    s = np.zeros(n_mod)
    _abi.check(lib().specula_mod_table_host(int(n_mod), c.ctypes.data_as(C.c_void_p),
                                            s.ctypes.data_as(C.c_void_p)),
               "specula_mod_table_host")
    return c, s


def specula_pupil_mask(ctx, pupil, amp, stream=None):
    import torch
    _abi.check(lib().specula_pupil_mask(
        ctx.handle, C.byref(pupil), _dev(amp, torch.float32, pupil.n_pix ** 2, "amp"),
        _stream(stream)), "specula_pupil_mask")


def specula_valid_subaps(ctx, pupil, n_sub, idx, n_valid, stream=None):
    import torch
    _abi.check(lib().specula_valid_subaps(
        ctx.handle, C.byref(pupil), int(n_sub), _dev(idx, torch.int32, n_sub * n_sub, "idx"),
        _dev(n_valid, torch.int32, 1, "n_valid"), _stream(stream)), "specula_valid_subaps")


# ---- screens ------------------------------------------------------------------------

def specula_screen_generate(ctx, side, pitch_m, r0_m, L0_m, noise, noise_sub, screen,
                            stream=None):
    """noise: CUDA complex128 (side, side) tensor; noise_sub: (3, 3, 3) complex
    array (host); screen: CUDA float32 (side, side) output."""
    import torch
    sub = np.ascontiguousarray(np.asarray(noise_sub, dtype=np.complex128))
    if sub.size != 27:
        raise ValueError("noise_sub must hold 3*3*3 complex values")
    _abi.check(lib().specula_screen_generate(
        ctx.handle, int(side), float(pitch_m), float(r0_m), float(L0_m),
        _dev(noise, torch.complex128, side * side, "noise"), sub.ctypes.data_as(C.c_void_p),
        _dev(screen, torch.float32, side * side, "screen"), _stream(stream)),
        "specula_screen_generate")


# ---- per-frame calls -----------------------------------------------------------------

def specula_atmo_extract(ctx, layers, screens, source, pupil, t, phase, t_dev=None,
                         stream=None):
    import torch
    n = len(layers)
    if len(screens) != n:
        raise ValueError("one screen per layer")
    L = (LayerDesc * n)(*layers)
    ptrs = (C.c_void_p * n)(*[C.c_void_p(s.data_ptr()) for s in screens])
    for s, l in zip(screens, layers):
        _dev(s, torch.float32, l.side * l.side, "screen")
    _abi.check(lib().specula_atmo_extract(
        ctx.handle, n, L, ptrs, C.byref(source), C.byref(pupil), float(t),
        _dev(t_dev, torch.float64, 1, "t_dev"),
        _dev(phase, torch.float32, pupil.n_pix ** 2, "phase"), _stream(stream)),
        "specula_atmo_extract")


def specula_rng_complex(ctx, seed, sample0, n_samples, stream_id, n_per_sample, out,
                        stream=None):
    import torch
    _abi.check(lib().specula_rng_complex(
        ctx.handle, int(seed), int(sample0), int(n_samples), int(stream_id), int(n_per_sample),
        _dev(out, torch.complex128, n_samples * n_per_sample, "out"), _stream(stream)),
        "specula_rng_complex")


def specula_screen_generate_batch(ctx, n_screens, side, pitch_m, r0_m, L0_m, seed, sample0,
                                  screens, stream=None):
    import torch
    _abi.check(lib().specula_screen_generate_batch(
        ctx.handle, int(n_screens), int(side), float(pitch_m), float(r0_m), float(L0_m),
        int(seed), int(sample0), _dev(screens, torch.float32, n_screens * side * side, "screens"),
        _stream(stream)), "specula_screen_generate_batch")


def specula_random_phase(ctx, screens, n, side, n_pix, scale, phase, stream=None):
    import torch
    _abi.check(lib().specula_random_phase(
        ctx.handle, _dev(screens, torch.float32, n * side * side, "screens"), int(n), int(side),
        int(n_pix), _dev(scale, torch.float32, n, "scale"),
        _dev(phase, torch.float32, n * n_pix * n_pix, "phase"), _stream(stream)),
        "specula_random_phase")


def specula_atmo_extract_noalloc(layers, screens, source, pupil, t, phase, t_dev=None,
                                 stream=None):
    """Context-free extraction for callers that cannot allocate device memory
    (see the header): same result as specula_atmo_extract."""
    import torch
    n = len(layers)
    if len(screens) != n:
        raise ValueError("one screen per layer")
    L = (LayerDesc * n)(*layers)
    ptrs = (C.c_void_p * n)(*[C.c_void_p(s.data_ptr()) for s in screens])
    for s, l in zip(screens, layers):
        _dev(s, torch.float32, l.side * l.side, "screen")
    _abi.check(lib().specula_atmo_extract_noalloc(
        n, L, ptrs, C.byref(source), C.byref(pupil), float(t),
        _dev(t_dev, torch.float64, 1, "t_dev"),
        _dev(phase, torch.float32, pupil.n_pix ** 2, "phase"), _stream(stream)),
        "specula_atmo_extract_noalloc")


def specula_pwfs_plan(ctx, pupil, pwfs):
    _abi.check(lib().specula_pwfs_plan(ctx.handle, C.byref(pupil), C.byref(pwfs)),
               "specula_pwfs_plan")


def specula_pwfs_set_slots(ctx, pupil, pwfs, slot_begin, slot_end):
    """Image only the modulation points of cosine slots [slot_begin, slot_end)."""
    _abi.check(lib().specula_pwfs_set_slots(ctx.handle, C.byref(pupil), C.byref(pwfs),
                                            int(slot_begin), int(slot_end)),
               "specula_pwfs_set_slots")


def specula_pwfs_set_form(ctx, pupil, pwfs, form):
    _abi.check(lib().specula_pwfs_set_form(ctx.handle, C.byref(pupil), C.byref(pwfs), int(form)),
               "specula_pwfs_set_form")


def specula_pwfs_set_tiles(ctx, pupil, pwfs, chunk, ka, passes=2):
    _abi.check(lib().specula_pwfs_set_tiles(ctx.handle, C.byref(pupil), C.byref(pwfs),
                                            int(chunk), int(ka), int(passes)),
               "specula_pwfs_set_tiles")


def specula_pwfs_get_tiles(ctx, pupil, pwfs):
    """(chunk, ka, passes) of the plan."""
    ch, ka, ps = C.c_int32(), C.c_int32(), C.c_int32()
    _abi.check(lib().specula_pwfs_get_tiles(ctx.handle, C.byref(pupil), C.byref(pwfs),
                                            C.byref(ch), C.byref(ka), C.byref(ps)),
               "specula_pwfs_get_tiles")
    return ch.value, ka.value, ps.value


def specula_pwfs_autotune(ctx, pupil, pwfs, amp, phase, det, reps=3,
                          max_workspace_bytes=512 << 20, stream=None):
    """Time the candidate tilings on these buffers, keep and return the best
    (chunk, ka, passes)."""
    import torch
    n = pupil.n_pix
    nb = phase.numel() // (n * n)
    side = pwfs.pad * pwfs.n_sub
    ch, ka, ps = C.c_int32(), C.c_int32(), C.c_int32()
    _abi.check(lib().specula_pwfs_autotune(
        ctx.handle, C.byref(pupil), C.byref(pwfs), _dev(amp, torch.float32, n * n, "amp"),
        _dev(phase, torch.float32, nb * n * n, "phase"), nb,
        _dev(det, torch.float32, nb * side * side, "det"), int(reps), int(max_workspace_bytes),
        C.byref(ch), C.byref(ka), C.byref(ps), _stream(stream)), "specula_pwfs_autotune")
    return ch.value, ka.value, ps.value


def specula_pwfs_image(ctx, pupil, pwfs, amp, phase, det, stream=None):
    """phase: (n_batch, n, n) or (n, n); det: (n_batch, 2 n_sub, 2 n_sub)."""
    import torch
    n = pupil.n_pix
    nb = phase.numel() // (n * n)
    side = pwfs.pad * pwfs.n_sub
    _abi.check(lib().specula_pwfs_image(
        ctx.handle, C.byref(pupil), C.byref(pwfs), _dev(amp, torch.float32, n * n, "amp"),
        _dev(phase, torch.float32, nb * n * n, "phase"), nb,
        _dev(det, torch.float32, nb * side * side, "det"), _stream(stream)),
        "specula_pwfs_image")


def _pwfs_at(pwfs, ratio):
    d = PwfsDesc(pwfs.pad, pwfs.n_mod, pwfs.n_sub, pwfs.pup_dist_px, pwfs.mod_amp * float(ratio))
    return d


def specula_pwfs_plan_poly(ctx, pupil, pwfs, ratios):
    """Plans for every wavelength of a polychromatic image (set-up)."""
    for r in ratios:
        specula_pwfs_plan(ctx, pupil, _pwfs_at(pwfs, r))


def specula_pwfs_image_poly(ctx, pupil, pwfs, ratios, weights, amp, phase, det, stream=None):
    """det = sum_i weights[i] image(phase * ratios[i], mod_amp * ratios[i]);
    ratios = lambda_ref / lambda_i."""
    import torch
    n = pupil.n_pix
    nb = phase.numel() // (n * n)
    side = pwfs.pad * pwfs.n_sub
    r = np.ascontiguousarray(ratios, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if r.shape != w.shape or r.ndim != 1:
        raise ValueError("ratios and weights must be 1-D of equal length")
    _abi.check(lib().specula_pwfs_image_poly(
        ctx.handle, C.byref(pupil), C.byref(pwfs), int(r.size), r.ctypes.data_as(C.c_void_p),
        w.ctypes.data_as(C.c_void_p), _dev(amp, torch.float32, n * n, "amp"),
        _dev(phase, torch.float32, nb * n * n, "phase"), nb,
        _dev(det, torch.float32, nb * side * side, "det"), _stream(stream)),
        "specula_pwfs_image_poly")


def specula_sh_plan(ctx, pupil, sh):
    nv = C.c_int32()
    _abi.check(lib().specula_sh_plan(ctx.handle, C.byref(pupil), C.byref(sh), C.byref(nv)),
               "specula_sh_plan")
    return nv.value


def specula_sh_image(ctx, pupil, sh, amp, phase, spots, n_valid, stream=None):
    import torch
    n = pupil.n_pix
    nb = phase.numel() // (n * n)
    _abi.check(lib().specula_sh_image(
        ctx.handle, C.byref(pupil), C.byref(sh), _dev(amp, torch.float32, n * n, "amp"),
        _dev(phase, torch.float32, nb * n * n, "phase"), nb,
        _dev(spots, torch.float32, nb * n_valid * sh.fft_n ** 2, "spots"), _stream(stream)),
        "specula_sh_image")


def specula_sh_image_poly(ctx, pupil, sh, ratios, weights, amp, phase, spots, n_valid,
                          stream=None):
    """spots = sum_i weights[i] ratios[i]^2 W_i spots(phase * ratios[i]) W_i^T,
    each wavelength's spots integrated over the reference pixels;
    ratios = lambda_ref / lambda_i."""
    import torch
    n = pupil.n_pix
    nb = phase.numel() // (n * n)
    r = np.ascontiguousarray(ratios, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if r.shape != w.shape or r.ndim != 1:
        raise ValueError("ratios and weights must be 1-D of equal length")
    _abi.check(lib().specula_sh_image_poly(
        ctx.handle, C.byref(pupil), C.byref(sh), int(r.size), r.ctypes.data_as(C.c_void_p),
        w.ctypes.data_as(C.c_void_p), _dev(amp, torch.float32, n * n, "amp"),
        _dev(phase, torch.float32, nb * n * n, "phase"), nb,
        _dev(spots, torch.float32, nb * n_valid * sh.fft_n ** 2, "spots"), _stream(stream)),
        "specula_sh_image_poly")


def specula_sh_set_range(ctx, pupil, sh, sub_begin, sub_end):
    """Image only the valid subapertures [sub_begin, sub_end) (set-up call)."""
    _abi.check(lib().specula_sh_set_range(ctx.handle, C.byref(pupil), C.byref(sh),
                                          int(sub_begin), int(sub_end)), "specula_sh_set_range")


def specula_slopes(ctx, slopec, img, ref, slopes, stream=None):
    import torch
    nb = slopes.numel() // (2 * slopec.n_valid)
    _abi.check(lib().specula_slopes(
        ctx.handle, C.byref(slopec), _dev(img, torch.float32, None, "img"),
        _dev(ref, torch.float32, 2 * slopec.n_valid, "ref"), nb,
        _dev(slopes, torch.float32, nb * 2 * slopec.n_valid, "slopes"), _stream(stream)),
        "specula_slopes")


def specula_recon(ctx, rec, slopes, modes, stream=None):
    import torch
    nb = slopes.numel() // rec.n_slopes
    _abi.check(lib().specula_recon(
        ctx.handle, C.byref(rec), _dev(slopes, torch.float32, nb * rec.n_slopes, "slopes"), nb,
        _dev(modes, torch.float32, nb * rec.n_modes, "modes"), _stream(stream)),
        "specula_recon")


def specula_ccd(ctx, det, scale, ron, seed, frame, out, frame_dev=None, stream=None):
    """out = Poisson(det scale) + ron N(0, 1), reproducible per (seed, frame);
    frame_dev (one int32 CUDA tensor, nullable) adds a device-side index."""
    import torch
    n = det.numel()
    _abi.check(lib().specula_ccd(
        ctx.handle, int(n), _dev(det, torch.float32, n, "det"), float(scale), float(ron),
        int(seed) & 0xFFFFFFFFFFFFFFFF, int(frame) & 0xFFFFFFFF,
        _dev(frame_dev, torch.int32, 1, "frame_dev"), _dev(out, torch.float32, n, "out"),
        _stream(stream)), "specula_ccd")


def specula_dm_shape(ctx, basis, cmd, phase, stream=None):
    """phase = B^T cmd: basis (n_modes, ...) float32, cmd (n_modes,), phase of
    the basis' trailing size."""
    import torch
    nm = basis.shape[0]
    npx = basis.numel() // nm
    _abi.check(lib().specula_dm_shape(
        ctx.handle, int(nm), int(npx), _dev(basis, torch.float32, nm * npx, "basis"),
        _dev(cmd, torch.float32, nm, "cmd"), _dev(phase, torch.float32, npx, "phase"),
        _stream(stream)), "specula_dm_shape")


def specula_loop_residual(ctx, amp, atm, dm, wfs_over_sci, resid, stats, stream=None):
    """resid = atm - dm; stats (2 float64) = (piston-free RMS, Strehl)."""
    import torch
    n = amp.numel()
    _abi.check(lib().specula_loop_residual(
        ctx.handle, int(n), _dev(amp, torch.float32, n, "amp"), _dev(atm, torch.float32, n, "atm"),
        _dev(dm, torch.float32, n, "dm"), float(wfs_over_sci),
        _dev(resid, torch.float32, n, "resid"), _dev(stats, torch.float64, 2, "stats"),
        _stream(stream)), "specula_loop_residual")


def specula_loop_integrate(ctx, gain, leak, modes, cmd, stream=None):
    """cmd = (1 - leak) cmd + gain modes."""
    import torch
    n = cmd.numel()
    _abi.check(lib().specula_loop_integrate(
        ctx.handle, int(n), float(gain), float(leak), _dev(modes, torch.float32, n, "modes"),
        _dev(cmd, torch.float32, n, "cmd"), _stream(stream)), "specula_loop_integrate")


def specula_fma_probe(ctx, bits, n_ctas, n_iter, sink, stream=None):
    """FMA-rate probe kernel (see the header); sink: n_ctas * 256 elements of
    float32 (bits 32) or float64 (bits 64)."""
    import torch
    dt = torch.float32 if bits == 32 else torch.float64
    _abi.check(lib().specula_fma_probe(ctx.handle, int(bits), int(n_ctas), int(n_iter),
                                       _dev(sink, dt, n_ctas * 256, "sink"), _stream(stream)),
               "specula_fma_probe")


def specula_rebin(ctx, img, n_out, out, stream=None):
    """Area-weighted rebinning of (..., n_in, n_in) images to (..., n_out, n_out)."""
    import torch
    n_in = img.shape[-1]
    nb = img.numel() // (n_in * n_in)
    _abi.check(lib().specula_rebin(ctx.handle, _dev(img, torch.float32, nb * n_in * n_in, "img"),
                                   int(n_in), int(n_out), int(nb),
                                   _dev(out, torch.float32, nb * n_out * n_out, "out"),
                                   _stream(stream)), "specula_rebin")


def specula_infscreen_operators(ctx, side, n_st, pitch_m, r0_m, L0_m, rcond=1e-12,
                                want_f64=False, stream=None):
    """(A [side, n_st side], B [side, side]) float32 operators of the line draw
    (plus their float64 copies when want_f64)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    A = torch.empty(side, n_st * side, device=dev)
    B = torch.empty(side, side, device=dev)
    A64 = torch.empty(side, n_st * side, dtype=torch.float64, device=dev) if want_f64 else None
    B64 = torch.empty(side, side, dtype=torch.float64, device=dev) if want_f64 else None
    _abi.check(lib().specula_infscreen_operators(
        ctx.handle, int(side), int(n_st), float(pitch_m), float(r0_m), float(L0_m), float(rcond),
        _dev(A), _dev(B), _dev(A64), _dev(B64), _stream(stream)), "specula_infscreen_operators")
    return (A, B, A64, B64) if want_f64 else (A, B)


def specula_infscreen_lines(ctx, side, n_st, tasks, seed=0, noise=None, stream=None):
    """One new line per task; tasks: (screen, A, B, b_scale, axis, direction,
    stream_id, line) tuples with distinct screens."""
    import torch
    if len(tasks) > INF_MAX_TASKS:
        raise ValueError(f"at most {INF_MAX_TASKS} tasks per call")
    arr = (InfLine * max(len(tasks), 1))()
    for i, (scr, A, B, bs, axis, direction, sid, line) in enumerate(tasks):
        arr[i] = InfLine(_dev(scr, torch.float32, side * side, "screen").value,
                         _dev(A, torch.float32, side * side * n_st, "A").value,
                         _dev(B, torch.float32, side * side, "B").value,
                         float(bs), int(axis), int(direction), int(sid), int(line))
    nz = _dev(noise, torch.float32, len(tasks) * side, "noise")
    _abi.check(lib().specula_infscreen_lines(ctx.handle, int(side), int(n_st), len(tasks),
                                             C.cast(arr, C.c_void_p), C.c_uint64(seed), nz,
                                             _stream(stream)), "specula_infscreen_lines")


def specula_infscreen_advance(ctx, layers, source, pupil, side, n_st, margin, screens, A, B,
                              b_scale, lo, t, seed=0, stream=None):
    """Plan and grow one frame's lines; lo (list of 2 n_layers ints) is
    updated in place; returns the number of kernel calls.  A, B: one operator
    tensor per layer."""
    import torch
    n = len(layers)
    L = (LayerDesc * max(n, 1))(*layers)
    lo_a = (C.c_int64 * max(2 * n, 1))(*lo)
    scr = (C.c_void_p * max(n, 1))(*[_dev(x, torch.float32, side * side, "screen").value
                                     for x in screens])
    Ap = (C.c_void_p * max(n, 1))(*[_dev(x, torch.float32, side * side * n_st, "A").value
                                    for x in A])
    Bp = (C.c_void_p * max(n, 1))(*[_dev(x, torch.float32, side * side, "B").value for x in B])
    bs = (C.c_float * max(n, 1))(*[float(x) for x in b_scale])
    calls = C.c_int32()
    _abi.check(lib().specula_infscreen_advance(
        ctx.handle, n, C.cast(L, C.c_void_p), C.byref(source), C.byref(pupil), int(side),
        int(n_st), int(margin), C.cast(scr, C.c_void_p), C.cast(Ap, C.c_void_p),
        C.cast(Bp, C.c_void_p), C.cast(bs, C.c_void_p), C.cast(lo_a, C.c_void_p), float(t),
        C.c_uint64(seed), C.byref(calls), _stream(stream)), "specula_infscreen_advance")
    lo[:] = list(lo_a[:2 * n])
    return calls.value


def specula_infscreen_plan(layers, source, pupil, side, margin, t, lo, max_moves=4096):
    """Host-only ring planner: (moves [(layer, axis, direction, line)], new lo).
    layers: LayerDesc list; lo: list of 2 n_layers ints (rows, columns per
    layer)."""
    n = len(layers)
    L = (LayerDesc * max(n, 1))(*layers)
    lo_a = (C.c_int64 * max(2 * n, 1))(*lo)
    mv = (InfMove * max(max_moves, 1))()
    nm = C.c_int32()
    _abi.check(lib().specula_infscreen_plan(n, C.cast(L, C.c_void_p), C.byref(source),
                                            C.byref(pupil), int(side), int(margin), float(t),
                                            C.cast(lo_a, C.c_void_p), int(max_moves),
                                            C.cast(mv, C.c_void_p), C.byref(nm)),
               "specula_infscreen_plan")
    return ([(m.layer, m.axis, m.direction, m.line) for m in mv[:nm.value]],
            list(lo_a[:2 * n]))


def specula_recon_reserve(ctx, rec, max_batch):
    """Size the workspace of rec's batched bf16 products for batches up to
    max_batch (set-up call)."""
    _abi.check(lib().specula_recon_reserve(ctx.handle, C.byref(rec), int(max_batch)),
               "specula_recon_reserve")


def specula_sh_poly_reserve(ctx, pupil, sh, max_batch):
    """Size the polychromatic SH workspace for batches up to max_batch (set-up
    call)."""
    _abi.check(lib().specula_sh_poly_reserve(ctx.handle, C.byref(pupil), C.byref(sh),
                                             int(max_batch)), "specula_sh_poly_reserve")


def specula_recon_convert(ctx, R, precision, hi, lo=None, stream=None):
    import torch
    nm, ns = R.shape
    _abi.check(lib().specula_recon_convert(
        ctx.handle, int(nm), int(ns), _dev(R, torch.float32, nm * ns, "R"), int(precision),
        _dev(hi, None, nm * ns, "hi"), _dev(lo, None, nm * ns, "lo"), _stream(stream)),
        "specula_recon_convert")


def specula_gemm_bf16(ctx, A, B, C, splits=1, work=None, stream=None):
    """C (M, N) float32 = A (M, K) bf16 @ B (N, K)^T bf16 on the tensor cores."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must share K")
    _abi.check(lib().specula_gemm_bf16(
        ctx.handle, _dev(A, torch.bfloat16, M * K, "A"), _dev(B, torch.bfloat16, N * K, "B"),
        int(M), int(N), int(K), _dev(C, torch.float32, M * N, "C"), int(splits),
        _dev(work, torch.float32, None, "work"), _stream(stream)), "specula_gemm_bf16")


def specula_gemm_tf32(ctx, A, B, C, splits=1, work=None, stream=None):
    """C (M, N) float32 = A (M, K) @ B (N, K)^T with tf32 operands (float32
    storage) on the tensor cores."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must share K")
    _abi.check(lib().specula_gemm_tf32(
        ctx.handle, _dev(A, torch.float32, M * K, "A"), _dev(B, torch.float32, N * K, "B"),
        int(M), int(N), int(K), _dev(C, torch.float32, M * N, "C"), int(splits),
        _dev(work, torch.float32, None, "work"), _stream(stream)), "specula_gemm_tf32")


def specula_col_stats(ctx, X, mean, std, stream=None):
    import torch
    R, Cc = X.shape
    _abi.check(lib().specula_col_stats(
        ctx.handle, _dev(X, torch.float32, R * Cc, "X"), int(R), int(Cc),
        _dev(mean, torch.float32, Cc, "mean"), _dev(std, torch.float32, Cc, "std"),
        _stream(stream)), "specula_col_stats")


def specula_affine_cols(ctx, X, shift, mul, out, stream=None):
    import torch
    R, Cc = X.shape
    _abi.check(lib().specula_affine_cols(
        ctx.handle, _dev(X, torch.float32, R * Cc, "X"), int(R), int(Cc),
        _dev(shift, torch.float32, Cc, "shift"), _dev(mul, torch.float32, Cc, "mul"),
        _dev(out, torch.float32, R * Cc, "out"), _stream(stream)), "specula_affine_cols")


class MLP:
    """Learned reconstructor handle (specula_mlp_*)."""

    def __init__(self, ctx, sizes, batch_max):
        n_in, h1, h2, n_out = sizes
        h = C.c_void_p()
        _abi.check(lib().specula_mlp_create(ctx.handle, int(n_in), int(h1), int(h2), int(n_out),
                                            int(batch_max), C.byref(h)), "specula_mlp_create")
        self.handle, self.sizes = h, tuple(sizes)
        ctx._children.add(self)

    def close(self):
        if self.handle:
            lib().specula_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layer(self, l, W, b):
        W = np.ascontiguousarray(W, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        assert W.shape == (self.sizes[l + 1], self.sizes[l]) and b.shape == (self.sizes[l + 1],)
        _abi.check(lib().specula_mlp_set_layer(self.handle, int(l), W.ctypes.data_as(C.c_void_p),
                                               b.ctypes.data_as(C.c_void_p)),
                   "specula_mlp_set_layer")

    def _get(self, fn, l, name):
        W = np.zeros((self.sizes[l + 1], self.sizes[l]), dtype=np.float32)
        b = np.zeros(self.sizes[l + 1], dtype=np.float32)
        _abi.check(fn(self.handle, int(l), W.ctypes.data_as(C.c_void_p),
                      b.ctypes.data_as(C.c_void_p)), name)
        return W, b

    def get_layer(self, l):
        return self._get(lib().specula_mlp_get_layer, l, "specula_mlp_get_layer")

    def get_grad(self, l):
        return self._get(lib().specula_mlp_get_grad, l, "specula_mlp_get_grad")

    def forward(self, X, Y=None, stream=None):
        import torch
        B = X.shape[0]
        _abi.check(lib().specula_mlp_forward(
            self.handle, _dev(X, torch.float32, B * self.sizes[0], "X"), int(B),
            _dev(Y, torch.float32, B * self.sizes[3], "Y"), _stream(stream)),
            "specula_mlp_forward")

    def infer(self, X, Y, stream=None):
        """Inference only (specula_mlp_infer): the weight-streaming path for
        batch <= 4, the forward pass otherwise."""
        import torch
        B = X.shape[0]
        _abi.check(lib().specula_mlp_infer(
            self.handle, _dev(X, torch.float32, B * self.sizes[0], "X"), int(B),
            _dev(Y, torch.float32, B * self.sizes[3], "Y"), _stream(stream)),
            "specula_mlp_infer")

    def backward(self, T, loss=None, stream=None):
        import torch
        B = T.shape[0]
        _abi.check(lib().specula_mlp_backward(
            self.handle, _dev(T, torch.float32, B * self.sizes[3], "T"), int(B),
            _dev(loss, torch.float32, 1, "loss"), _stream(stream)), "specula_mlp_backward")

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        _abi.check(lib().specula_mlp_adam(self.handle, float(lr), float(b1), float(b2),
                                          float(eps), _stream(stream)), "specula_mlp_adam")


def specula_mlp_create(ctx, n_in, n_h1, n_h2, n_out, batch_max):
    return MLP(ctx, (n_in, n_h1, n_h2, n_out), batch_max)


def specula_mlp_destroy(mlp):
    mlp.close()


def specula_mlp_set_layer(mlp, layer, W, b):
    mlp.set_layer(layer, W, b)


def specula_mlp_get_layer(mlp, layer):
    return mlp.get_layer(layer)


def specula_mlp_get_grad(mlp, layer):
    return mlp.get_grad(layer)


def specula_mlp_forward(mlp, X, Y=None, stream=None):
    mlp.forward(X, Y, stream)


def specula_mlp_infer(mlp, X, Y, stream=None):
    mlp.infer(X, Y, stream)


def specula_mlp_backward(mlp, T, loss=None, stream=None):
    mlp.backward(T, loss, stream)


def specula_mlp_adam(mlp, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    mlp.adam(lr, b1, b2, eps, stream)


def specula_modal_basis_host(pupil, n_modes):
    out = np.zeros((n_modes, pupil.n_pix, pupil.n_pix))
    _abi.check(lib().specula_modal_basis_host(C.byref(pupil), int(n_modes),
                                              out.ctypes.data_as(C.c_void_p)),
               "specula_modal_basis_host")
    return out


def specula_modal_basis(ctx, pupil, n_modes, basis, stream=None):
    import torch
    _abi.check(lib().specula_modal_basis(
        ctx.handle, C.byref(pupil), int(n_modes),
        _dev(basis, torch.float32, n_modes * pupil.n_pix ** 2, "basis"), _stream(stream)),
        "specula_modal_basis")


def specula_calib_intmat(ctx, pupil, pwfs, amp, basis, n_modes, push_amp, slopec, im,
                         stream=None):
    import torch
    _abi.check(lib().specula_calib_intmat(
        ctx.handle, C.byref(pupil), C.byref(pwfs), _dev(amp, torch.float32, pupil.n_pix ** 2, "amp"),
        _dev(basis, torch.float32, n_modes * pupil.n_pix ** 2, "basis"), int(n_modes),
        float(push_amp), C.byref(slopec),
        _dev(im, torch.float64, 2 * slopec.n_valid * n_modes, "im"), _stream(stream)),
        "specula_calib_intmat")


def specula_pinv_fp64(ctx, A, rcond, R, R32=None, stream=None):
    """A: (m, n) float64 CUDA tensor; R: (n, m) float64 output.  Returns rank."""
    import torch
    m, n = A.shape
    rk = C.c_int32()
    _abi.check(lib().specula_pinv_fp64(
        ctx.handle, _dev(A, torch.float64, m * n, "A"), int(m), int(n), float(rcond),
        _dev(R, torch.float64, m * n, "R"), _dev(R32, torch.float32, m * n, "R32"),
        C.byref(rk), _stream(stream)), "specula_pinv_fp64")
    return rk.value


def slopec_desc(kind, n_sub, idx_dev, fft_n=0):
    import torch
    _dev(idx_dev, torch.int32, None, "subap_idx")
    nv = idx_dev.numel() // 4 if kind == SLOPES_PYR_MAPS else idx_dev.numel()
    d = SlopecDesc(int(kind), int(n_sub), int(nv), int(fft_n), C.c_void_p(idx_dev.data_ptr()))
    d._keep = (idx_dev,)          # the descriptor holds a raw pointer: keep the tensor alive
    return d


def recon_desc(n_modes, n_slopes, precision, R_dev, R_lo_dev=None):
    import torch
    want = torch.float32 if precision == PREC_FP32 else (torch.int16, torch.bfloat16,
                                                          torch.uint16)
    for t in (R_dev, R_lo_dev):
        if t is None:
            continue
        ok = t.dtype == want if precision == PREC_FP32 else t.dtype in want
        if not ok or not t.is_cuda or not t.is_contiguous() or t.numel() < n_modes * n_slopes:
            raise ValueError(f"reconstructor tensor must be a contiguous CUDA tensor of "
                             f"{n_modes}x{n_slopes} {want}, got {t.dtype} {tuple(t.shape)}")
    d = ReconDesc(int(n_modes), int(n_slopes), int(precision), C.c_void_p(R_dev.data_ptr()),
                  C.c_void_p(R_lo_dev.data_ptr()) if R_lo_dev is not None else None)
    d._keep = (R_dev, R_lo_dev)   # the descriptor holds raw pointers: keep the tensors alive
    return d


# ---- multi-sensor system in one persistent launch -----------------------------------
WFS_PYR, WFS_SH = 0, 1
MWFS_PHASE, MWFS_DETECTOR = 0, 1


def wfs_desc(sensor):
    """WfsDesc from a workload sensor (kind 'pwfs' or 'sh')."""
    d = WfsDesc()
    d.pupil = pupil_desc(sensor.pupil)
    d.source = source_desc(sensor.source)
    if sensor.kind == "pwfs":
        d.kind = WFS_PYR
        d.pwfs = pwfs_desc(sensor.pwfs)
    elif sensor.kind == "sh":
        d.kind = WFS_SH
        g = sensor.sh
        d.sh = ShDesc(g.n_sub, g.sub_pix, g.fft_n)
    else:
        raise ValueError(sensor.kind)
    return d


class Mwfs:
    """Multi-sensor system (specula_mwfs_*): every sensor, the slopes and the
    reconstructor product in one persistent launch per frame.  Keeps
    references to the screens and R, whose device memory the library uses."""

    def __init__(self, ctx, sensors, layers, screens, R=None):
        import torch
        descs = (WfsDesc * len(sensors))(*sensors)
        lds = (LayerDesc * len(layers))(*layers)
        for t in screens:
            _dev(t, torch.float32, None, "screen")
        ptrs = (C.c_void_p * len(screens))(*[t.data_ptr() for t in screens])
        n_modes = 0 if R is None else int(R.shape[0])
        h = C.c_void_p()
        _abi.check(lib().specula_mwfs_create(
            ctx.handle, len(sensors), descs, len(layers), lds, ptrs, n_modes,
            _dev(R, torch.float32, None, "R"), C.byref(h)), "specula_mwfs_create")
        self.handle = h
        self._keep = (list(screens), R)
        self.n_sensors, self.n_modes = len(sensors), n_modes
        tot = C.c_int32()
        _abi.check(lib().specula_mwfs_info(h, -1, None, None, C.byref(tot)), "specula_mwfs_info")
        self.n_slopes = tot.value
        if R is not None and R.shape[1] != self.n_slopes:
            self.close()
            raise ValueError(f"R must have {self.n_slopes} columns")
        self.n_valid, self.slope_offset = [], []
        for k in range(len(sensors)):
            nv, off = C.c_int32(), C.c_int32()
            _abi.check(lib().specula_mwfs_info(h, k, C.byref(nv), C.byref(off), None),
                       "specula_mwfs_info")
            self.n_valid.append(nv.value)
            self.slope_offset.append(off.value)
        ctx._children.add(self)

    def close(self):
        if self.handle:
            lib().specula_mwfs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def schedule(self):
        nt, g, mg = C.c_int32(), C.c_int32(), C.c_int32()
        _abi.check(lib().specula_mwfs_schedule(self.handle, C.byref(nt), C.byref(g), C.byref(mg)),
                   "specula_mwfs_schedule")
        return {"n_tasks": nt.value, "grid": g.value, "max_grid": mg.value}

    def set_grid(self, ctas):
        _abi.check(lib().specula_mwfs_set_grid(self.handle, int(ctas)), "specula_mwfs_set_grid")

    def set_wait(self, limit_ns=0, stall_task=-1):
        _abi.check(lib().specula_mwfs_set_wait(self.handle, int(limit_ns), int(stall_task)),
                   "specula_mwfs_set_wait")

    def frame(self, t, slopes, modes=None, ref=None, t_dev=None, stream=None):
        import torch
        _abi.check(lib().specula_mwfs_frame(
            self.handle, float(t), _dev(t_dev, torch.float64, 1, "t_dev"),
            _dev(ref, torch.float32, self.n_slopes, "ref"),
            _dev(slopes, torch.float32, self.n_slopes, "slopes"),
            _dev(modes, torch.float32, self.n_modes, "modes"), _stream(stream)),
            "specula_mwfs_frame")

    def reference(self, ref, modes=None, stream=None):
        import torch
        _abi.check(lib().specula_mwfs_reference(
            self.handle, _dev(ref, torch.float32, self.n_slopes, "ref"),
            _dev(modes, torch.float32, self.n_modes, "modes"), _stream(stream)),
            "specula_mwfs_reference")

    def read(self, sensor, what, dst, stream=None):
        import torch
        _abi.check(lib().specula_mwfs_read(self.handle, int(sensor), int(what),
                                           _dev(dst, torch.float32, None, "dst"), _stream(stream)),
                   "specula_mwfs_read")


def specula_mwfs_create(ctx, sensors, layers, screens, R=None):
    return Mwfs(ctx, sensors, layers, screens, R)


def specula_mwfs_destroy(m):
    m.close()


def specula_mwfs_frame(m, t, slopes, modes=None, ref=None, t_dev=None, stream=None):
    m.frame(t, slopes, modes, ref, t_dev, stream)


def specula_mwfs_reference(m, ref, modes=None, stream=None):
    m.reference(ref, modes, stream)


def specula_mwfs_read(m, sensor, what, dst, stream=None):
    m.read(sensor, what, dst, stream)


def specula_mwfs_info(m):
    return {"n_valid": list(m.n_valid), "slope_offset": list(m.slope_offset),
            "n_slopes": m.n_slopes}


def specula_mwfs_schedule(m):
    return m.schedule()


def specula_mwfs_set_grid(m, ctas):
    m.set_grid(ctas)


def specula_mwfs_set_wait(m, limit_ns, stall_task):
    m.set_wait(limit_ns, stall_task)
