"""ctypes binding of librtseg.so: the C ABI declared in include/rt.h, with the
same function names. Argument marshalling only -- every step of the path runs
in the library's CUDA kernels. Importing this module raises if the library has
not been built: there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtseg.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ETIMEOUT, RT_EMARKER, RT_EQUEUE, RT_EUNAVAIL, RT_ESIZE = range(9)
RT_AUTO, RT_RASTER, RT_QUEUE, RT_HYBRID, RT_FRONTIER = range(5)

# every symbol declared in include/rt.h
EXPORTS = (
    "rt_create", "rt_destroy", "rt_status_str", "rt_version", "rt_workspace_bytes", "rt_marker",
    "rt_reconstruct", "rt_fill_holes", "rt_label_area", "rt_edt", "rt_seg_params_default",
    "rt_segment_batch", "rt_timing_enable", "rt_timing_read", "rt_kernel_launches", "rt_recon_stats",
    "rt_edt_noalloc", "rt_synth_tile", "rt_tile_features", "rt_mlp_forward", "rt_mlp_forward_tc", "rt_mlp_backward", "rt_mlp_backward_tc",
    "rt_mlp_adamw", "rt_set_picker", "rt_last_picks", "rt_set_limits", "rt_segment_workspace_bytes",
    "rt_feature_norm", "rt_watershed", "rt_object_features", "rt_set_picker_classes", "rt_set_queue_capacity",
)
RT_NPHASES = 9
PHASES = ("recon_init", "recon_sweep", "recon_out", "fill", "label", "edt", "pick", "objects", "watershed")
RT_NOBJFEAT = 20
RT_NFEATURES = 24
RT_MLP_NPARAM = 5955
RT_POLICY_PLAIN, RT_POLICY_LEARNED = 0, 1

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_int = ctypes.c_int


class RtTile(ctypes.Structure):
    _fields_ = [
        ("img", _vp), ("ld_img", _i64), ("H", _int), ("W", _int),
        ("recon", _vp), ("ld_recon", _i64),
        ("filled", _vp), ("ld_filled", _i64),
        ("labels", _vp), ("ld_labels", _i64),
        ("d2", _vp), ("ld_d2", _i64),
        ("n_kept", _vp), ("status", _vp),
    ]


class RtSegParams(ctypes.Structure):
    _fields_ = [(n, _int) for n in ("h_offset", "threshold", "min_area", "max_area", "conn_recon",
                                    "conn_fill", "variant", "max_local", "policy", "max_iters", "timeout_ms",
                                    "pick_min_prob", "strip_tiles")]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"librtseg.so is not built ({path}); run paper_1405_7958_gb300/build.py")
    lib = ctypes.CDLL(path)
    lib.rt_create.argtypes = [ctypes.POINTER(_vp), _int, ctypes.c_size_t]
    lib.rt_create.restype = _int
    lib.rt_set_limits.argtypes = [_vp, _int, _int]
    lib.rt_set_limits.restype = _int
    lib.rt_destroy.argtypes = [_vp]
    lib.rt_destroy.restype = None
    lib.rt_status_str.argtypes = [_int]
    lib.rt_status_str.restype = ctypes.c_char_p
    lib.rt_version.argtypes = []
    lib.rt_version.restype = _int
    lib.rt_workspace_bytes.argtypes = [_vp]
    lib.rt_workspace_bytes.restype = ctypes.c_size_t
    lib.rt_marker.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp]
    lib.rt_marker.restype = _int
    lib.rt_reconstruct.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _int, _int, _int, _int, _int, _vp, _vp]
    lib.rt_reconstruct.restype = _int
    lib.rt_fill_holes.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _vp]
    lib.rt_fill_holes.restype = _int
    lib.rt_label_area.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _i32, _i32, _vp, _vp, _vp]
    lib.rt_label_area.restype = _int
    lib.rt_edt.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _vp, _vp]
    lib.rt_edt.restype = _int
    lib.rt_watershed.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _int, _vp, _i64, _vp, _vp, _vp]
    lib.rt_watershed.restype = _int
    lib.rt_object_features.argtypes = [_vp, _vp, _i64, _vp, _i64, _int, _int, _vp, _vp, _int, _vp, _vp, _vp]
    lib.rt_object_features.restype = _int
    lib.rt_edt_noalloc.argtypes = [_vp, _i64, _vp, _i64, _int, _int, _vp, _vp]
    lib.rt_edt_noalloc.restype = _int
    lib.rt_synth_tile.argtypes = [_vp, _vp, _i64, _int, _int, ctypes.c_uint64] + [_int] * 10 + [_vp]
    lib.rt_synth_tile.restype = _int
    lib.rt_tile_features.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_int),
                                     ctypes.POINTER(_int), _int, _vp, _vp]
    lib.rt_tile_features.restype = _int
    lib.rt_mlp_forward.argtypes = [_vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, ctypes.c_float, _int, _vp]
    lib.rt_mlp_forward.restype = _int
    lib.rt_mlp_forward_tc.argtypes = [_vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, ctypes.c_float, _int, _vp, _vp]
    lib.rt_mlp_forward_tc.restype = _int
    lib.rt_mlp_backward_tc.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, _vp]
    lib.rt_mlp_backward_tc.restype = _int
    lib.rt_mlp_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _int, _vp, _vp, _vp]
    lib.rt_mlp_backward.restype = _int
    _f = ctypes.c_float
    lib.rt_mlp_adamw.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _int, _f, _f, _f, _f, _f, _vp]
    lib.rt_mlp_adamw.restype = _int
    lib.rt_set_picker.argtypes = [_vp, _vp, _vp]
    lib.rt_set_picker.restype = _int
    lib.rt_set_picker_classes.argtypes = [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]
    lib.rt_set_picker_classes.restype = _int
    lib.rt_last_picks.argtypes = [_vp, ctypes.POINTER(_int), _int]
    lib.rt_last_picks.restype = _int
    lib.rt_seg_params_default.argtypes = [ctypes.POINTER(RtSegParams)]
    lib.rt_seg_params_default.restype = None
    lib.rt_segment_batch.argtypes = [_vp, ctypes.POINTER(RtTile), _int, ctypes.POINTER(RtSegParams), _vp]
    lib.rt_segment_batch.restype = _int
    lib.rt_segment_workspace_bytes.argtypes = [_vp, ctypes.POINTER(RtTile), _int, ctypes.POINTER(RtSegParams)]
    lib.rt_segment_workspace_bytes.restype = ctypes.c_size_t
    lib.rt_set_queue_capacity.argtypes = [_vp, _i64]
    lib.rt_set_queue_capacity.restype = _int
    lib.rt_feature_norm.argtypes = [_vp, _vp, _int, _vp, _vp]
    lib.rt_feature_norm.restype = _int
    lib.rt_timing_enable.argtypes = [_vp, _int]
    lib.rt_timing_enable.restype = _int
    lib.rt_timing_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _int]
    lib.rt_timing_read.restype = _int
    lib.rt_kernel_launches.argtypes = [_vp]
    lib.rt_kernel_launches.restype = _i64
    lib.rt_recon_stats.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    lib.rt_recon_stats.restype = _int
    return lib
