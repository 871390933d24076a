"""ctypes binding of libgs.so (the C ABI in include/gs.h).

Argument marshalling only: every function here forwards to the library of
the same name.  Loading fails loudly if the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GS_CHECKED=1 selects the checked build (index checks that report instead of
# faulting; build.build(checked=True))
LIB_PATH = os.path.join(HERE, "libgs_checked.so" if os.environ.get("GS_CHECKED") == "1" else "libgs.so")

GS_TILE = 16
GS_MAX_VIEWS = 64
GS_FLAG_ZERO_ACCUM = 1
GS_FLAG_EXTENT_3SIGMA = 2
GS_FLAG_MASK_BITS = 4
GS_SELFTEST_SCRATCH_BYTES = 4096
GS_ERR_TIMEOUT = 4

STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
          4: "GS_ERR_TIMEOUT", 5: "GS_ERR_DEVICE_CHECK"}


class GsError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("znear", C.c_float), ("lowpass", C.c_float), ("clamp", C.c_float),
                ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("t_min", C.c_float),
                ("bg", C.c_float * 3), ("flags", C.c_uint32)]


class Scene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("rotations", C.c_void_p),
                ("opacities", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("sh_coeffs", C.c_int32)]


class Plan(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_items", C.c_int64), ("total_pixels", C.c_int64),
                ("n_entries", C.c_int64), ("n_views", C.c_int32), ("total_tiles", C.c_int32),
                ("sort_bits", C.c_int32), ("n_pairs", C.c_int32),
                ("cams", Camera * GS_MAX_VIEWS), ("tile_base", C.c_int32 * (GS_MAX_VIEWS + 1)),
                ("pixel_base", C.c_int64 * (GS_MAX_VIEWS + 1))]


class SceneBuf(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("rotations", C.c_void_p),
                ("opacities", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("sh_coeffs", C.c_int32)]


class FwdOutputs(C.Structure):
    _fields_ = [("image", C.c_void_p), ("final_T", C.c_void_p), ("n_contrib", C.c_void_p),
                ("imax", C.c_void_p), ("wmax", C.c_void_p), ("depth", C.c_void_p),
                ("depth_blend", C.c_void_p), ("weight_sum", C.c_void_p), ("max_area", C.c_void_p),
                ("weight_sum_fixed", C.c_void_p), ("depth_center", C.c_void_p), ("n_blended", C.c_void_p)]


class Grads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_scales", C.c_void_p), ("d_rotations", C.c_void_p),
                ("d_opacities", C.c_void_p), ("d_sh", C.c_void_p), ("d_mean2d_abs", C.c_void_p),
                ("weight_sum", C.c_void_p), ("weight_sum_fixed", C.c_void_p)]


class PreprocessView(C.Structure):
    _fields_ = [("xy_tau_z", C.c_void_p), ("conic_o", C.c_void_p), ("rgb", C.c_void_p),
                ("tiles", C.c_void_p), ("rect", C.c_void_p), ("sorted_items", C.c_void_p),
                ("offsets", C.c_void_p), ("pair_offsets", C.c_void_p)]


class SortView(C.Structure):
    _fields_ = [("tile_ids", C.c_void_p), ("items", C.c_void_p), ("ranges", C.c_void_p)]


class ConfigIdentify(C.Structure):
    _fields_ = [("theta_blur", C.c_float), ("keep_visible", C.c_float), ("keep_critical", C.c_float)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char_p), ("ms", C.c_double), ("launches", C.c_int64)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "gs_config_default": (None, [C.POINTER(Config)]),
    "gs_plan_init": (C.c_int, [C.POINTER(Plan), C.c_int64, C.POINTER(Camera), C.c_int32]),
    "gs_preprocess_workspace_size": (C.c_size_t, [C.POINTER(Plan)]),
    "gs_bin_sort_workspace_size": (C.c_size_t, [C.POINTER(Plan)]),
    "gs_preprocess": (C.c_int, [C.POINTER(Plan), C.POINTER(Scene), C.POINTER(Config), C.c_void_p,
                                C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_pack_mask": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]),
    "gs_bin_sort": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_render_fwd": (C.c_int, [C.POINTER(Plan), C.POINTER(Config), C.c_void_p, C.c_void_p,
                                C.POINTER(FwdOutputs), C.c_void_p]),
    "gs_render_bwd": (C.c_int, [C.POINTER(Plan), C.POINTER(Scene), C.POINTER(Config), C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Grads),
                                C.c_void_p]),
    "gs_bin_sort_noalloc": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "gs_prune_workspace_size": (C.c_size_t, [C.c_int64]),
    "gs_prune_select": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "gs_gather_scene": (C.c_int, [C.POINTER(Scene), C.c_void_p, C.c_int64, C.POINTER(SceneBuf), C.c_void_p]),
    "gs_config_identify_default": (None, [C.POINTER(ConfigIdentify)]),
    "gs_identify_workspace_size": (C.c_size_t, [C.POINTER(Plan)]),
    "gs_identify": (C.c_int, [C.POINTER(Plan), C.POINTER(ConfigIdentify), C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                              C.c_void_p]),
    "gs_clone_gaussians": (C.c_int, [C.POINTER(Scene), C.c_void_p, C.c_int64, C.POINTER(SceneBuf), C.c_void_p]),
    "gs_sample_workspace_size": (C.c_size_t, [C.c_int64]),
    "gs_sample_gaussians": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_depth_points_workspace_size": (C.c_size_t, [C.POINTER(Plan)]),
    "gs_depth_points": (C.c_int, [C.POINTER(Plan), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_size_t, C.c_void_p]),
    "gs_loss_l1_ssim_workspace_size": (C.c_size_t, [C.POINTER(Plan)]),
    "gs_loss_l1_ssim": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_loss_l1": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gs_selftest_wait_timeout": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p]),
    "gs_device_status": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.c_void_p]),
    "gs_inspect_preprocess": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.POINTER(PreprocessView)]),
    "gs_inspect_sort": (C.c_int, [C.POINTER(Plan), C.c_void_p, C.POINTER(SortView)]),
    "gs_timing_enable": (C.c_int, [C.c_int]),
    "gs_timing_collect": (C.c_int, [C.POINTER(KernelTime), C.c_int]),
    "gs_status_string": (C.c_char_p, [C.c_int]),
    "gs_sizeof_plan": (C.c_size_t, []),
    "gs_sizeof_camera": (C.c_size_t, []),
    "gs_sizeof_config": (C.c_size_t, []),
    "gs_sizeof_scene": (C.c_size_t, []),
}

_LIB = None


def lib() -> C.CDLL:
    """The loaded libgs.so, with argument types set.  Raises if missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        for name, cls in (("gs_sizeof_plan", Plan), ("gs_sizeof_camera", Camera),
                          ("gs_sizeof_config", Config), ("gs_sizeof_scene", Scene)):
            if getattr(L, name)() != C.sizeof(cls):
                raise RuntimeError(f"ABI mismatch for {name}")
        _LIB = L
    return _LIB


def check(fn: str, status: int) -> None:
    if status != 0:
        raise GsError(fn, status)
