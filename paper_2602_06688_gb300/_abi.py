"""ctypes declarations of the C ABI in include/specula_gb300.h.

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspecula_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ENONFINITE, ENOPLAN = \
    0, -1, -2, -3, -4, -5, -6, -7
SLOPES_PYR, SLOPES_SH, SLOPES_PYR_MAPS = 0, 1, 2
PWFS_FORM_TILT, PWFS_FORM_SHIFTED, PWFS_FORM_DFTGEMM_BF16, PWFS_FORM_DFTGEMM_TF32 = 0, 1, 2, 3
PREC_FP32, PREC_BF16, PREC_BF16X2 = 0, 1, 2


class PupilDesc(C.Structure):
    _fields_ = [("n_pix", C.c_int32), ("pitch_m", C.c_double),
                ("obsc_frac", C.c_double)]


class SourceDesc(C.Structure):
    _fields_ = [("theta_x_rad", C.c_double), ("theta_y_rad", C.c_double),
                ("height_m", C.c_double), ("wavelength_nm", C.c_double)]


class LayerDesc(C.Structure):
    _fields_ = [("side", C.c_int32), ("pitch_m", C.c_double),
                ("height_m", C.c_double), ("vx_mps", C.c_double),
                ("vy_mps", C.c_double)]


class PwfsDesc(C.Structure):
    _fields_ = [("pad", C.c_int32), ("n_mod", C.c_int32), ("n_sub", C.c_int32),
                ("pup_dist_px", C.c_int32), ("mod_amp", C.c_double)]


class ShDesc(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("sub_pix", C.c_int32),
                ("fft_n", C.c_int32)]


class SlopecDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_sub", C.c_int32),
                ("n_valid", C.c_int32), ("fft_n", C.c_int32),
                ("subap_idx_dev", C.c_void_p)]


class WfsDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pupil", PupilDesc), ("source", SourceDesc),
                ("pwfs", PwfsDesc), ("sh", ShDesc)]


class ReconDesc(C.Structure):
    _fields_ = [("n_modes", C.c_int32), ("n_slopes", C.c_int32),
                ("precision", C.c_int32), ("R_dev", C.c_void_p),
                ("R_lo_dev", C.c_void_p)]


class InfLine(C.Structure):
    _fields_ = [("screen_dev", C.c_void_p), ("A_dev", C.c_void_p), ("B_dev", C.c_void_p),
                ("b_scale", C.c_float), ("axis", C.c_int32), ("direction", C.c_int32),
                ("stream_id", C.c_int32), ("line", C.c_int64)]


class InfMove(C.Structure):
    _fields_ = [("layer", C.c_int32), ("axis", C.c_int32), ("direction", C.c_int32),
                ("line", C.c_int64)]


INF_MAX_TASKS = 32

P = C.POINTER
vp = C.c_void_p
i32 = C.c_int32
dbl = C.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "specula_strerror": (C.c_char_p, [C.c_int]),
    "specula_last_cuda_error": (C.c_char_p, []),
    "specula_version": (C.c_int, []),
    "specula_ctx_create": (C.c_int, [P(vp), C.c_int]),
    "specula_ctx_destroy": (C.c_int, [vp]),
    "specula_ctx_status": (C.c_int, [vp, P(i32)]),
    "specula_ctx_set_guard": (C.c_int, [vp, i32]),
    "specula_check_guards": (C.c_int, [vp, P(i32), P(i32)]),
    "specula_prof_enable": (C.c_int, [vp, i32]),
    "specula_prof_read": (C.c_int, [vp, vp, vp]),
    "specula_launch_count": (C.c_int, [vp, P(C.c_int64)]),
    "specula_graph_begin": (C.c_int, [vp, vp]),
    "specula_graph_end": (C.c_int, [vp, vp, P(vp)]),
    "specula_graph_launch": (C.c_int, [vp, vp]),
    "specula_graph_kernel_count": (C.c_int, [vp, P(C.c_int64)]),
    "specula_graph_destroy": (C.c_int, [vp]),
    "specula_pupil_mask_host": (C.c_int, [P(PupilDesc), vp]),
    "specula_valid_subaps_host": (C.c_int, [P(PupilDesc), i32, vp, P(i32)]),
    "specula_mod_table_host": (C.c_int, [i32, vp, vp]),
    "specula_pupil_mask": (C.c_int, [vp, P(PupilDesc), vp, vp]),
    "specula_valid_subaps": (C.c_int, [vp, P(PupilDesc), i32, vp, vp, vp]),
    "specula_screen_generate": (C.c_int, [vp, i32, dbl, dbl, dbl, vp, vp, vp, vp]),
    "specula_atmo_extract": (C.c_int, [vp, i32, P(LayerDesc), P(vp), P(SourceDesc),
                                       P(PupilDesc), dbl, vp, vp, vp]),
    "specula_rng_complex": (C.c_int, [vp, C.c_uint64, i32, i32, i32, C.c_int64, vp, vp]),
    "specula_screen_generate_batch": (C.c_int, [vp, i32, i32, dbl, dbl, dbl, C.c_uint64, i32,
                                                vp, vp]),
    "specula_random_phase": (C.c_int, [vp, vp, i32, i32, i32, vp, vp, vp]),
    "specula_atmo_extract_noalloc": (C.c_int, [i32, P(LayerDesc), P(vp), P(SourceDesc),
                                               P(PupilDesc), dbl, vp, vp, vp]),
    "specula_pwfs_plan": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc)]),
    "specula_pwfs_set_tiles": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), i32, i32, i32]),
    "specula_pwfs_set_form": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), i32]),
    "specula_pwfs_set_slots": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), i32, i32]),
    "specula_pyr_image_index_host": (C.c_int, [P(PupilDesc), i32, i32, i32, vp, P(i32)]),
    "specula_pwfs_image_poly": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), i32, vp, vp, vp, vp, i32,
                                          vp, vp]),
    "specula_dm_shape": (C.c_int, [vp, i32, i32, vp, vp, vp, vp]),
    "specula_ccd": (C.c_int, [vp, i32, vp, C.c_double, C.c_double, C.c_uint64, C.c_uint32, vp,
                              vp, vp]),
    "specula_loop_residual": (C.c_int, [vp, i32, vp, vp, vp, C.c_double, vp, vp, vp]),
    "specula_loop_integrate": (C.c_int, [vp, i32, C.c_float, C.c_float, vp, vp, vp]),
    "specula_infscreen_operators": (C.c_int, [vp, i32, i32, dbl, dbl, dbl, dbl, vp, vp, vp, vp,
                                              vp]),
    "specula_rebin": (C.c_int, [vp, vp, i32, i32, i32, vp, vp]),
    "specula_fma_probe": (C.c_int, [vp, i32, i32, i32, vp, vp]),
    "specula_infscreen_lines": (C.c_int, [vp, i32, i32, i32, vp, C.c_uint64, vp, vp]),
    "specula_infscreen_plan": (C.c_int, [i32, vp, P(SourceDesc), P(PupilDesc), i32, i32, dbl, vp,
                                         i32, vp, P(i32)]),
    "specula_infscreen_advance": (C.c_int, [vp, i32, vp, P(SourceDesc), P(PupilDesc), i32, i32,
                                            i32, vp, vp, vp, vp, vp, dbl, C.c_uint64, P(i32),
                                            vp]),
    "specula_pwfs_get_tiles": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), P(i32), P(i32),
                                         P(i32)]),
    "specula_pwfs_autotune": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), vp, vp, i32, vp, i32,
                                        C.c_int64, P(i32), P(i32), P(i32), vp]),
    "specula_pwfs_image": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), vp, vp, i32, vp, vp]),
    "specula_sh_plan": (C.c_int, [vp, P(PupilDesc), P(ShDesc), P(i32)]),
    "specula_sh_image": (C.c_int, [vp, P(PupilDesc), P(ShDesc), vp, vp, i32, vp, vp]),
    "specula_sh_image_poly": (C.c_int, [vp, P(PupilDesc), P(ShDesc), i32, vp, vp, vp, vp, i32,
                                        vp, vp]),
    "specula_sh_set_range": (C.c_int, [vp, P(PupilDesc), P(ShDesc), i32, i32]),
    "specula_slopes": (C.c_int, [vp, P(SlopecDesc), vp, vp, i32, vp, vp]),
    "specula_recon": (C.c_int, [vp, P(ReconDesc), vp, i32, vp, vp]),
    "specula_recon_convert": (C.c_int, [vp, i32, i32, vp, i32, vp, vp, vp]),
    "specula_recon_reserve": (C.c_int, [vp, P(ReconDesc), i32]),
    "specula_sh_poly_reserve": (C.c_int, [vp, P(PupilDesc), P(ShDesc), i32]),
    "specula_gemm_bf16": (C.c_int, [vp, vp, vp, i32, i32, i32, vp, i32, vp, vp]),
    "specula_gemm_tf32": (C.c_int, [vp, vp, vp, i32, i32, i32, vp, i32, vp, vp]),
    "specula_col_stats": (C.c_int, [vp, vp, i32, i32, vp, vp, vp]),
    "specula_affine_cols": (C.c_int, [vp, vp, C.c_int64, i32, vp, vp, vp, vp]),
    "specula_mlp_create": (C.c_int, [vp, i32, i32, i32, i32, i32, P(vp)]),
    "specula_mlp_destroy": (C.c_int, [vp]),
    "specula_mlp_set_layer": (C.c_int, [vp, i32, vp, vp]),
    "specula_mlp_get_layer": (C.c_int, [vp, i32, vp, vp]),
    "specula_mlp_get_grad": (C.c_int, [vp, i32, vp, vp]),
    "specula_mlp_forward": (C.c_int, [vp, vp, i32, vp, vp]),
    "specula_mlp_backward": (C.c_int, [vp, vp, i32, vp, vp]),
    "specula_mlp_infer": (C.c_int, [vp, vp, i32, vp, vp]),
    "specula_mlp_adam": (C.c_int, [vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]),
    "specula_modal_basis_host": (C.c_int, [P(PupilDesc), i32, vp]),
    "specula_modal_basis": (C.c_int, [vp, P(PupilDesc), i32, vp, vp]),
    "specula_calib_intmat": (C.c_int, [vp, P(PupilDesc), P(PwfsDesc), vp, vp, i32, dbl,
                                       P(SlopecDesc), vp, vp]),
    "specula_pinv_fp64": (C.c_int, [vp, vp, i32, i32, dbl, vp, vp, P(i32), vp]),
    "specula_mwfs_create": (C.c_int, [vp, i32, P(WfsDesc), i32, P(LayerDesc), P(vp), i32, vp,
                                      P(vp)]),
    "specula_mwfs_destroy": (C.c_int, [vp]),
    "specula_mwfs_info": (C.c_int, [vp, i32, P(i32), P(i32), P(i32)]),
    "specula_mwfs_schedule": (C.c_int, [vp, P(i32), P(i32), P(i32)]),
    "specula_mwfs_set_grid": (C.c_int, [vp, i32]),
    "specula_mwfs_set_wait": (C.c_int, [vp, C.c_int64, i32]),
    "specula_mwfs_frame": (C.c_int, [vp, dbl, vp, vp, vp, vp, vp]),
    "specula_mwfs_reference": (C.c_int, [vp, vp, vp, vp]),
    "specula_mwfs_read": (C.c_int, [vp, i32, i32, vp, vp]),
}

_lib = None


def load():
    """Load libspecula_gb300.so (built by ``build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with "
            "paper_2602_06688_gb300.build.build() (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SpeculaError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        text = lib.specula_strerror(status).decode()
        if status == ECUDA:
            detail = lib.specula_last_cuda_error().decode()
            if detail:
                text += f": {detail}"
        super().__init__(f"{where}: {text} ({status})")
        self.status = status


def check(status, where):
    if status != OK:
        raise SpeculaError(status, where)
    return status
