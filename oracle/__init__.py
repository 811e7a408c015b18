"""CPU oracle for the segmentation hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations (in ``oracle.c``) of the
operations that the paper's segmentation stage runs as GPU tasks
(Section 5.1 "Example Application": ReconToNuclei, FillHoles, Pre-Watershed,
BWLabel; Section 3.2.1: AreaThreshold). Only ``tests/``, the smoke check and
the CPU-baseline leg of ``bench.py`` may import this package; the GPU product
path never does, and it shares no code with the CUDA sources.

The C library is compiled with gcc on first use (or by ``build()``); nothing
here needs a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_OBJ = os.path.join(_HERE, "objects.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, -O2, no vector intrinsics)."""
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in (_SRC, _SRC_OBJ))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_OBJ, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_marker.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.orc_marker.restype = None
            lib.orc_recon_fixpoint.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               _u8p, _i64p]
            lib.orc_recon_vincent.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.orc_threshold_below.argtypes = [_u8p, ctypes.c_long, ctypes.c_int, _u8p]
            lib.orc_threshold_below.restype = None
            lib.orc_fill_holes.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.orc_label_area.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _i32p, _i32p]
            lib.orc_edt_brute.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _i32p]
            lib.orc_edt_meijster.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _i32p]
            lib.orc_edt_at.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_edt_at.restype = ctypes.c_int64
            lib.orc_object_features.argtypes = [_i32p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p,
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
            lib.orc_watershed.argtypes = [_i32p, _i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p,
                                          ctypes.POINTER(ctypes.c_int)]
            lib.orc_chain.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _u8p, _u8p, _i32p, _i32p, _i32p]
            _lib = lib
    return _lib


def _u8(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8 or a.ndim != 2:
        raise TypeError("expected a 2-D uint8 array")
    return a


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def marker(I: np.ndarray, h: int = 30) -> np.ndarray:
    """J = max(I - h, 0) inside, J = I on the one-pixel border."""
    I = _u8(I)
    J = np.empty_like(I)
    _load().orc_marker(_p(I, _u8p), I.shape[0], I.shape[1], int(h), _p(J, _u8p))
    return J


def recon_fixpoint(J: np.ndarray, I: np.ndarray, conn: int = 8, return_iters: bool = False):
    """Reconstruction by dilation as its definition: iterate R <- min(delta(R), I)
    from R = min(J, I) until nothing changes (slow; small images)."""
    J, I = _u8(J), _u8(I)
    if J.shape != I.shape:
        raise ValueError("shape mismatch")
    R = np.empty_like(I)
    it = ctypes.c_long(0)
    _check(_load().orc_recon_fixpoint(_p(J, _u8p), _p(I, _u8p), I.shape[0], I.shape[1], conn,
                                      _p(R, _u8p), ctypes.byref(it)), "recon_fixpoint")
    return (R, it.value) if return_iters else R


def recon(J: np.ndarray, I: np.ndarray, conn: int = 8) -> np.ndarray:
    """Reconstruction by dilation by Vincent's hybrid algorithm (same result
    as recon_fixpoint, fast enough for 4K x 4K)."""
    J, I = _u8(J), _u8(I)
    if J.shape != I.shape:
        raise ValueError("shape mismatch")
    R = np.empty_like(I)
    _check(_load().orc_recon_vincent(_p(J, _u8p), _p(I, _u8p), I.shape[0], I.shape[1], conn,
                                     _p(R, _u8p)), "recon_vincent")
    return R


def threshold_below(R: np.ndarray, t: int = 80) -> np.ndarray:
    R = _u8(R)
    B = np.empty_like(R)
    _load().orc_threshold_below(_p(R, _u8p), R.size, int(t), _p(B, _u8p))
    return B


def fill_holes(B: np.ndarray, conn: int = 4) -> np.ndarray:
    """1 on foreground and on background not conn-connected to the border."""
    B = _u8(B)
    F = np.empty_like(B)
    _check(_load().orc_fill_holes(_p(B, _u8p), B.shape[0], B.shape[1], conn, _p(F, _u8p)), "fill_holes")
    return F


def label_area(F: np.ndarray, min_area: int = 20, max_area: int = 1000, conn: int = 8,
               return_count: bool = False):
    """Component labels = smallest linear index of the component; -1 on the
    background and on components with area outside [min_area, max_area]."""
    F = _u8(F)
    L = np.empty(F.shape, dtype=np.int32)
    n = ctypes.c_int32(0)
    _check(_load().orc_label_area(_p(F, _u8p), F.shape[0], F.shape[1], conn, int(min_area),
                                  int(max_area), _p(L, _i32p), ctypes.byref(n)), "label_area")
    return (L, n.value) if return_count else L


def edt_brute(fg: np.ndarray) -> np.ndarray:
    """Squared EDT by brute force over all background pixels (tiny images)."""
    fg = _u8(fg)
    D = np.empty(fg.shape, dtype=np.int32)
    _check(_load().orc_edt_brute(_p(fg, _u8p), fg.shape[0], fg.shape[1], _p(D, _i32p)), "edt_brute")
    return D


def edt_at(fg: np.ndarray, r: int, c: int) -> int:
    """Squared EDT of one pixel by brute force (-1 if there is no background)."""
    fg = _u8(fg)
    return int(_load().orc_edt_at(_p(fg, _u8p), fg.shape[0], fg.shape[1], int(r), int(c)))


def edt(fg: np.ndarray) -> np.ndarray:
    """Squared EDT by Meijster's separable algorithm (int64 inside)."""
    fg = _u8(fg)
    D = np.empty(fg.shape, dtype=np.int32)
    _check(_load().orc_edt_meijster(_p(fg, _u8p), fg.shape[0], fg.shape[1], _p(D, _i32p)), "edt")
    return D


def chain(I: np.ndarray, h: int = 30, conn_recon: int = 8, t: int = 80, conn_fill: int = 4,
          min_area: int = 20, max_area: int = 1000):
    """The whole segmentation chain; returns dict(R, F, L, D, n_kept)."""
    I = _u8(I)
    H, W = I.shape
    R = np.empty_like(I)
    F = np.empty_like(I)
    L = np.empty((H, W), dtype=np.int32)
    D = np.empty((H, W), dtype=np.int32)
    n = ctypes.c_int32(0)
    _check(_load().orc_chain(_p(I, _u8p), H, W, int(h), int(conn_recon), int(t), int(conn_fill),
                             int(min_area), int(max_area), _p(R, _u8p), _p(F, _u8p), _p(L, _i32p),
                             _p(D, _i32p), ctypes.byref(n)), "chain")
    return {"R": R, "F": F, "L": L, "D": D, "n_kept": n.value}


NFEAT = 20
FEATURE_NAMES = ("area", "perimeter", "bbox_h", "bbox_w", "centroid_r", "centroid_c", "major_axis", "minor_axis",
                 "eccentricity", "compactness", "mean", "std", "min", "max", "median", "entropy", "glcm_pairs",
                 "glcm_contrast", "glcm_energy", "glcm_homogeneity")
# features whose values are integers (compared exactly)
INTEGER_FEATURES = (0, 1, 2, 3, 12, 13, 14, 16)


def _i32(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.int32 or a.ndim != 2:
        raise TypeError("expected a 2-D int32 array")
    return a


def object_features(L: np.ndarray, I: np.ndarray):
    """Per-object features of the label image L (>= 0: object label) over the
    intensities I: (labels ascending, float64 n x 20). See objects.c."""
    L, I = _i32(L), _u8(I)
    if L.shape != I.shape:
        raise ValueError("shape mismatch")
    n = ctypes.c_int(0)
    _check(_load().orc_object_features(_p(L, _i32p), _p(I, _u8p), L.shape[0], L.shape[1], 0, None, None,
                                       ctypes.byref(n)), "object_features")
    labels = np.empty(max(n.value, 1), dtype=np.int32)
    feat = np.empty((max(n.value, 1), NFEAT), dtype=np.float64)
    _check(_load().orc_object_features(_p(L, _i32p), _p(I, _u8p), L.shape[0], L.shape[1], n.value,
                                       _p(labels, _i32p), feat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(n)), "object_features")
    return labels[:n.value], feat[:n.value]


def watershed(L: np.ndarray, D: np.ndarray, h: int = 2, return_count: bool = False):
    """Marker-controlled watershed of the distance map D inside every object
    of L (basin label per object pixel, -1 elsewhere). See objects.c."""
    L, D = _i32(L), _i32(D)
    if L.shape != D.shape:
        raise ValueError("shape mismatch")
    B = np.empty_like(L)
    n = ctypes.c_int(0)
    _check(_load().orc_watershed(_p(L, _i32p), _p(D, _i32p), L.shape[0], L.shape[1], int(h), _p(B, _i32p),
                                 ctypes.byref(n)), "watershed")
    return (B, n.value) if return_count else B
