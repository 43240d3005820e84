"""GB300 (sm_103a) fast Hough transform: thin Python binding of libfht.so.

Every function here marshals arguments to the C ABI declared in
``include/fht.h`` and returns the output tensor; all arithmetic runs in the
library's CUDA kernels. PyTorch supplies device memory and streams only. If the
compiled library is missing, importing this package raises ImportError: there
is no CPU fallback.

The transform is Brady's dyadic fast Hough transform as used by Aliev,
Ershov and Nikolaev (arXiv:1811.06378): quadrants of the Hough image
(Section 3.1), the full four-quadrant image (Section 3.3), the angle-range
variant (Section 4) and fhtshift (Section 5), plus the adjoint.
"""

from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

__all__ = [
    "Q0", "Q1", "Q2", "Q3", "LAYOUT_QUADRANT", "LAYOUT_FULL", "FHTError", "lib",
    "query_shape", "full_shape", "full_row_to_quadrant", "angle_to_slopes",
    "workspace_size", "forward", "forward_range", "full_quadrants", "fhtshift",
    "adjoint", "FHTFunction", "profile_begin", "profile_end", "launch_count", "device_status",
    "workspace_size_many", "forward_many", "adjoint_many",
    "workspace_size_sheared", "shear_range", "forward_sheared",
    "scaled_width", "scaled_shape", "workspace_size_scaled", "scale_range", "forward_scaled",
    "workspace_size_padded", "forward_padded", "merge_strips",
    "BatchPlan", "FHT_OK", "FHT_ETIMEOUT", "FHT_EBOUNDS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
# FHT_DEBUG=1 loads the bounds-checked build (python -m
# paper_1811_06378_gb300.build --debug): every global access of the pass
# kernels is checked against the pass's buffers; device_status() reports
# FHT_EBOUNDS for any refused access.
DEBUG = os.environ.get("FHT_DEBUG") == "1"
LIB_PATH = os.path.join(_HERE, "_build", "debug" if DEBUG else "", "libfht.so")

Q0, Q1, Q2, Q3 = 0, 1, 2, 3
LAYOUT_QUADRANT, LAYOUT_FULL = 0, 1
FHT_OK, FHT_ETIMEOUT, FHT_EBOUNDS = 0, 5, 6
_U8, _I32, _F32 = 0, 1, 2
_DTYPE = {torch.uint8: _U8, torch.int32: _I32, torch.float32: _F32}


class FHTError(RuntimeError):
    """A libfht call returned a status other than FHT_OK."""


class Tuning(ctypes.Structure):
    """fht_tuning: levels fused per pass and tile widths for 2^K-row quadrants."""
    _fields_ = [("max_levels", ctypes.c_int), ("tile_u8", ctypes.c_int),
                ("tile_wide", ctypes.c_int)]


class BatchedTuning(ctypes.Structure):
    """fht_batched_tuning: how batched plans cut their work."""
    _fields_ = [("units_per_item", ctypes.c_int), ("tile_u8", ctypes.c_int),
                ("tile_wide", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("first_levels", ctypes.c_int * 13)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        how = ("python -m paper_1811_06378_gb300.build --debug" if DEBUG else
               "python -c 'import __graft_entry__ as g; g.build()'")
        raise ImportError(f"{LIB_PATH} is not built; run `{how}` (needs nvcc for sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    sz = ctypes.c_size_t
    sigs = {
        "fht_status_string": (ctypes.c_char_p, [i]),
        "fht_last_cuda_error": (i, []),
        "fht_query_shape": (i, [i, i, i, ip, ip]),
        "fht_full_shape": (i, [i, i, ip, ip]),
        "fht_full_row_to_quadrant": (i, [i, i, i, ip, ip]),
        "fht_angle_to_slopes": (i, [d, d, i, i, ip, ip]),
        "fht_workspace_size": (i, [i, i, i, i, i, i, ctypes.POINTER(sz)]),
        "fht_forward": (i, [vp, i, i, i, i64, i, vp, i, i64, vp, sz, vp]),
        "fht_forward_range": (i, [vp, i, i, i, i64, i, i, i, vp, i, i64, vp, sz, vp]),
        "fht_full_quadrants": (i, [vp, i, i, i, i64, vp, i, i64, i, vp, sz, vp]),
        "fhtshift": (i, [vp, vp, i, i, i, i, i, i, i64, i64, vp]),
        "fht_adjoint": (i, [vp, i, i, i, i, i, i64, vp, i64, vp, sz, vp]),
        "fht_workspace_size_sheared": (i, [i, i, i, i, i, ctypes.POINTER(sz)]),
        "fht_segment": (i, [i, i, i, i, i, i, i, ip, ip, ip, ip, ip]),
        "fht_forward_op": (i, [vp, i, i, i, i64, i, i, i, i, vp, i, i64, vp, sz, vp]),
        "fht_row_argmax": (i, [vp, i, i, i, i64, vp, vp, vp]),
        "fht_forward_sheared": (i, [vp, i, i, i, i64, i, d, i, i, vp, i, i64, vp, sz, vp]),
        "fht_shear_range": (i, [d, d, i, i, ip, ctypes.POINTER(d), ip, ip]),
        "fht_scaled_width": (i, [i, d, ip]),
        "fht_scaled_shape": (i, [i, i, i, d, ip, ip]),
        "fht_workspace_size_scaled": (i, [i, i, i, d, i, i, ctypes.POINTER(sz)]),
        "fht_forward_scaled": (i, [vp, i, i, i, i64, i, d, d, i, i, vp, i, i64, vp, sz, vp]),
        "fht_scale_range": (i, [d, d, i, i, ip, ctypes.POINTER(d), ctypes.POINTER(d), ip, ip]),
        "fht_workspace_size_padded": (i, [i, i, i, i, i, i, i, ctypes.POINTER(sz)]),
        "fht_forward_padded": (i, [vp, i, i, i, i64, i, i, i, vp, i, i64, vp, sz, vp]),
        "fht_merge_strips": (i, [vp, i, i, i, i, i64, i64, i, i, vp, i64, vp]),
        "fht_plan_create_batched": (i, [ctypes.POINTER(i), ctypes.POINTER(i), i, i, i, i,
                                        ctypes.POINTER(vp), ctypes.POINTER(sz)]),
        "fht_forward_batched": (i, [vp, vp, vp, sz, vp]),
        "fht_adjoint_batched": (i, [vp, vp, vp, sz, vp]),
        "fht_batched_status": (i, [vp, vp, vp]),
        "fht_batched_test_hooks": (i, [vp, ctypes.c_longlong, i]),
        "fht_plan_destroy": (None, [vp]),
        "fht_profile_begin": (i, []),
        "fht_profile_end": (i, [vp, i, ip]),
        "fht_launch_count": (ctypes.c_longlong, []),
        "fht_device_status": (ctypes.c_int, []),
        "fht_debug_test_hooks": (ctypes.c_int, [ctypes.c_longlong]),
        "fht_workspace_size_many": (i, [i, i, i, i, i, ctypes.POINTER(sz)]),
        "fht_forward_many": (i, [vp, i, i64, i, i, i64, i, i, vp, i64, i64, vp, sz, vp]),
        "fht_adjoint_many": (i, [vp, i, i64, i, i, i, i, i64, vp, i64, i64, vp, sz, vp]),
    }
    sigs["fht_set_tuning"] = (i, [i, ctypes.POINTER(Tuning)])
    sigs["fht_get_tuning"] = (i, [i, ctypes.POINTER(Tuning)])
    sigs["fht_set_batched_tuning"] = (i, [ctypes.POINTER(BatchedTuning)])
    sigs["fht_get_batched_tuning"] = (i, [ctypes.POINTER(BatchedTuning)])
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def _check(status: int, what: str) -> None:
    if status != 0:
        msg = lib.fht_status_string(status).decode()
        cuda = lib.fht_last_cuda_error()
        raise FHTError(f"{what}: {msg} (status {status}, last CUDA error {cuda})")


def _ints(k: int):
    return (ctypes.c_int * k)()


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev2d(t: torch.Tensor, name: str) -> tuple[int, int]:
    """(dtype code, pitch) of a row-major 2-D CUDA tensor."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit column stride")
    if t.dtype not in _DTYPE:
        raise ValueError(f"{name}: unsupported dtype {t.dtype}")
    return _DTYPE[t.dtype], max(t.stride(0), t.shape[1])


# ------------------------------------------------------------------ tuning

def set_tuning(K: int, max_levels: int | None = None, tile_u8: int = 1,
               tile_wide: int = 1) -> None:
    """Tuning for quadrants with 2^K rows from now on (fht_set_tuning);
    max_levels=None restores the default."""
    if max_levels is None:
        _check(lib.fht_set_tuning(K, None), "fht_set_tuning")
        return
    t = Tuning(max_levels, tile_u8, tile_wide)
    _check(lib.fht_set_tuning(K, ctypes.byref(t)), "fht_set_tuning")


def get_tuning(K: int) -> tuple[int, int, int]:
    """(max_levels, tile_u8, tile_wide) in use for 2^K-row quadrants."""
    t = Tuning()
    _check(lib.fht_get_tuning(K, ctypes.byref(t)), "fht_get_tuning")
    return t.max_levels, t.tile_u8, t.tile_wide


def set_batched_tuning(t: dict | None) -> None:
    """Tuning of batched plans created from now on (fht_set_batched_tuning):
    a dict with units_per_item, tile_u8, tile_wide, ctas_per_sm and
    first_levels ({K: levels}); missing keys keep their current values; None
    restores the defaults."""
    if t is None:
        _check(lib.fht_set_batched_tuning(None), "fht_set_batched_tuning")
        return
    cur = BatchedTuning()
    _check(lib.fht_get_batched_tuning(ctypes.byref(cur)), "fht_get_batched_tuning")
    for k in ("units_per_item", "tile_u8", "tile_wide", "ctas_per_sm"):
        if k in t:
            setattr(cur, k, int(t[k]))
    for K, f in (t.get("first_levels") or {}).items():
        cur.first_levels[int(K)] = int(f)
    _check(lib.fht_set_batched_tuning(ctypes.byref(cur)), "fht_set_batched_tuning")


def get_batched_tuning() -> dict:
    """The batched tuning in use, as set_batched_tuning takes it."""
    t = BatchedTuning()
    _check(lib.fht_get_batched_tuning(ctypes.byref(t)), "fht_get_batched_tuning")
    return {"units_per_item": t.units_per_item, "tile_u8": t.tile_u8,
            "tile_wide": t.tile_wide, "ctas_per_sm": t.ctas_per_sm,
            "first_levels": {K: t.first_levels[K] for K in range(7, 13)
                             if t.first_levels[K]}}


TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def load_tuning(path: str) -> dict:
    """Apply an autotuner table (JSON, see autotune.py) to the library."""
    with open(path) as f:
        res = json.load(f)
    for k, e in res["table"].items():
        set_tuning(int(k), int(e["max_levels"]), int(e["tile_u8"]), int(e["tile_wide"]))
    if "batched" in res:   # replaces the batched tuning in force
        set_batched_tuning(None)
        set_batched_tuning(res["batched"]["tuning"])
    return res


def _load_default_tuning() -> None:
    """The autotuner's table for this GPU (tuning_gb300.json), or the file
    FHT_TUNE_FILE names; FHT_TUNE_FILE=none keeps the library's defaults."""
    path = os.environ.get("FHT_TUNE_FILE")
    if path is None:
        path = TUNING_FILE if os.path.exists(TUNING_FILE) else None
    elif path.lower() == "none":
        path = None
    if path:
        load_tuning(path)


# ------------------------------------------------------------------ geometry

def query_shape(h: int, w: int, q: int) -> tuple[int, int]:
    r, c = ctypes.c_int(), ctypes.c_int()
    _check(lib.fht_query_shape(h, w, q, ctypes.byref(r), ctypes.byref(c)), "fht_query_shape")
    return r.value, c.value


def full_shape(h: int, w: int) -> tuple[int, int]:
    r, c = ctypes.c_int(), ctypes.c_int()
    _check(lib.fht_full_shape(h, w, ctypes.byref(r), ctypes.byref(c)), "fht_full_shape")
    return r.value, c.value


def full_row_to_quadrant(h: int, w: int, row: int) -> tuple[int, int]:
    q, t = ctypes.c_int(), ctypes.c_int()
    _check(lib.fht_full_row_to_quadrant(h, w, row, ctypes.byref(q), ctypes.byref(t)),
           "fht_full_row_to_quadrant")
    return q.value, t.value


def angle_to_slopes(phi_lo: float, phi_hi: float, h: int, w: int):
    lo, hi = _ints(4), _ints(4)
    _check(lib.fht_angle_to_slopes(phi_lo, phi_hi, h, w, lo, hi), "fht_angle_to_slopes")
    return list(lo), list(hi)


def workspace_size(h: int, w: int, layout: int, q: int, in_dtype: torch.dtype,
                   acc_dtype: torch.dtype) -> int:
    b = ctypes.c_size_t()
    _check(lib.fht_workspace_size(h, w, layout, q, _DTYPE[in_dtype], _DTYPE[acc_dtype],
                                  ctypes.byref(b)), "fht_workspace_size")
    return b.value


def _workspace(ws, nbytes: int, device) -> torch.Tensor | None:
    if nbytes == 0:
        return ws
    if ws is None:
        return torch.empty(nbytes, dtype=torch.uint8, device=device)
    if ws.numel() * ws.element_size() < nbytes:
        raise ValueError(f"workspace too small: need {nbytes} bytes")
    return ws


def _shape(t: torch.Tensor, shape, name: str) -> None:
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _nbytes(t) -> int:
    return 0 if t is None else t.numel() * t.element_size()


# ------------------------------------------------------------------ forward

def forward(img: torch.Tensor, q: int = Q0, acc: torch.dtype = torch.int32,
            out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Quadrant q of the Hough image of img: (n, W) tensor of dtype acc."""
    it, ip = _dev2d(img, "img")
    h, w = img.shape
    n, W = query_shape(h, w, q)
    if out is None:
        out = torch.empty((n, W), dtype=acc, device=img.device)
    _shape(out, (n, W), "out")
    ot, op = _dev2d(out, "out")
    ws = _workspace(workspace, workspace_size(h, w, LAYOUT_QUADRANT, q, img.dtype, acc),
                    img.device)
    _check(lib.fht_forward(_ptr(img), it, h, w, ip, q, _ptr(out), ot, op, _ptr(ws),
                           _nbytes(ws), _stream(stream)), "fht_forward")
    return out


def forward_range(img: torch.Tensor, q: int, t_lo: int, t_hi: int,
                  acc: torch.dtype = torch.int32, out: torch.Tensor | None = None,
                  workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Slopes t_lo..t_hi of quadrant q: (t_hi - t_lo + 1, W) tensor."""
    it, ip = _dev2d(img, "img")
    h, w = img.shape
    n, W = query_shape(h, w, q)
    if out is None:
        out = torch.empty((max(t_hi - t_lo + 1, 0), W), dtype=acc, device=img.device)
    _shape(out, (t_hi - t_lo + 1, W), "out")
    ot, op = _dev2d(out, "out")
    ws = _workspace(workspace, workspace_size(h, w, LAYOUT_QUADRANT, q, img.dtype, acc),
                    img.device)
    _check(lib.fht_forward_range(_ptr(img), it, h, w, ip, q, t_lo, t_hi, _ptr(out), ot, op,
                                 _ptr(ws), _nbytes(ws), _stream(stream)), "fht_forward_range")
    return out


def full_quadrants(img: torch.Tensor, acc: torch.dtype = torch.int32,
                   apply_fhtshift: bool = False, out: torch.Tensor | None = None,
                   workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Full four-quadrant Hough image of img (Section 3.3)."""
    it, ip = _dev2d(img, "img")
    h, w = img.shape
    R, W = full_shape(h, w)
    if out is None:
        out = torch.empty((R, W), dtype=acc, device=img.device)
    _shape(out, (R, W), "out")
    ot, op = _dev2d(out, "out")
    ws = _workspace(workspace, workspace_size(h, w, LAYOUT_FULL, 0, img.dtype, acc),
                    img.device)
    _check(lib.fht_full_quadrants(_ptr(img), it, h, w, ip, _ptr(out), ot, op,
                                  int(bool(apply_fhtshift)), _ptr(ws), _nbytes(ws),
                                  _stream(stream)), "fht_full_quadrants")
    return out


def fhtshift(hough: torch.Tensor, h: int, w: int, layout: int = LAYOUT_FULL, q: int = Q0,
             inverse: bool = False, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """fhtshift (Section 5) of a quadrant or full Hough image of an h x w image."""
    t, ip = _dev2d(hough, "hough")
    expect = full_shape(h, w) if layout == LAYOUT_FULL else query_shape(h, w, q)
    _shape(hough, expect, "hough")
    if out is None:
        out = torch.empty_like(hough)
    _shape(out, expect, "out")
    ot, op = _dev2d(out, "out")
    if ot != t:
        raise ValueError("out must have the dtype of hough")
    _check(lib.fhtshift(_ptr(hough), _ptr(out), t, h, w, layout, q, int(bool(inverse)), ip,
                        op, _stream(stream)), "fhtshift")
    return out


def adjoint(grad: torch.Tensor, h: int, w: int, layout: int = LAYOUT_FULL, q: int = Q0,
            out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Adjoint of forward (layout QUADRANT) or full_quadrants (layout FULL)."""
    t, ip = _dev2d(grad, "grad")
    _shape(grad, full_shape(h, w) if layout == LAYOUT_FULL else query_shape(h, w, q), "grad")
    if out is None:
        out = torch.empty((h, w), dtype=grad.dtype, device=grad.device)
    _shape(out, (h, w), "out")
    ot, op = _dev2d(out, "out")
    if ot != t:
        raise ValueError("out must have the dtype of grad")
    ws = _workspace(workspace, workspace_size(h, w, layout, q, grad.dtype, grad.dtype),
                    grad.device)
    _check(lib.fht_adjoint(_ptr(grad), t, h, w, layout, q, ip, _ptr(out), op, _ptr(ws),
                           _nbytes(ws), _stream(stream)), "fht_adjoint")
    return out


# ------------------------------------------------------------------ batched

# ------------------------------------------------------------------ other operations

OP_SUM, OP_MAX, OP_MIN = 0, 1, 2


def forward_op(img: torch.Tensor, q: int, op: int, t_lo: int = 0, t_hi: int | None = None,
               acc: torch.dtype | None = None, out: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Slope rows t_lo..t_hi of quadrant q with the sum (OP_SUM), maximum
    (OP_MAX) or minimum (OP_MIN) along every pattern (fht_forward_op)."""
    it, ip = _dev2d(img, "img")
    h, w = img.shape
    n, W = query_shape(h, w, q)
    t_hi = n - 1 if t_hi is None else t_hi
    if acc is None:
        acc = torch.float32 if img.dtype == torch.float32 else torch.int32
    if out is None:
        out = torch.empty((t_hi - t_lo + 1, W), dtype=acc, device=img.device)
    _shape(out, (t_hi - t_lo + 1, W), "out")
    ot, op_ = _dev2d(out, "out")
    ws = _workspace(workspace, workspace_size(h, w, LAYOUT_QUADRANT, q, img.dtype, out.dtype),
                    img.device)
    _check(lib.fht_forward_op(_ptr(img), it, h, w, ip, q, op, t_lo, t_hi, _ptr(out), ot, op_,
                              _ptr(ws), _nbytes(ws), _stream(stream)), "fht_forward_op")
    return out


# ------------------------------------------------------------------ back to lines

def segment(h: int, w: int, row: int, col: int, layout: int = LAYOUT_FULL, q: int = Q0,
            shifted: bool = False):
    """The image segment Hough point (row, col) sums (Section 3.2):
    (count, (r0, c0), (r1, c1)), or None when it lies wholly in the padding."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib.fht_segment(h, w, layout, q, row, col, int(shifted),
                           *[ctypes.byref(x) for x in v]), "fht_segment")
    if v[0].value == 0:
        return None
    return v[0].value, (v[1].value, v[2].value), (v[3].value, v[4].value)


def row_argmax(hough: torch.Tensor, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """(max, first argmax) of every row of a 2-D int32/float32 CUDA tensor."""
    code, pitch = _dev2d(hough, "hough")
    rows, cols = hough.shape
    vals = torch.empty(rows, dtype=hough.dtype, device=hough.device)
    idx = torch.empty(rows, dtype=torch.int32, device=hough.device)
    _check(lib.fht_row_argmax(_ptr(hough), code, rows, cols, pitch, _ptr(vals), _ptr(idx),
                              _stream(stream)), "fht_row_argmax")
    return vals, idx


# ------------------------------------------------------------------ sheared (Section 4)

def workspace_size_sheared(h: int, w: int, q: int, in_dtype: torch.dtype,
                           acc: torch.dtype) -> int:
    n = ctypes.c_size_t()
    _check(lib.fht_workspace_size_sheared(h, w, q, _DTYPE[in_dtype], _DTYPE[acc],
                                          ctypes.byref(n)), "fht_workspace_size_sheared")
    return n.value


def shear_range(phi_lo: float, phi_hi: float, h: int, w: int) -> tuple[int, float, int, int]:
    """(q, spl, t_lo, t_hi): the one sheared quadrant and its slope rows for
    the line angles [phi_lo, phi_hi] degrees (fht_shear_range)."""
    q, t_lo, t_hi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    spl = ctypes.c_double()
    _check(lib.fht_shear_range(phi_lo, phi_hi, h, w, ctypes.byref(q), ctypes.byref(spl),
                               ctypes.byref(t_lo), ctypes.byref(t_hi)), "fht_shear_range")
    return q.value, spl.value, t_lo.value, t_hi.value


def forward_sheared(img: torch.Tensor, q: int, spl: float, t_lo: int = 0,
                    t_hi: int | None = None, acc: torch.dtype = torch.int32,
                    out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Rows t_lo..t_hi of quadrant q of the image sheared by spl per row
    (Section 4; fht_forward_sheared)."""
    in_code, in_pitch = _dev2d(img, "img")
    h, w = img.shape
    n, W = query_shape(h, w, q)
    t_hi = n - 1 if t_hi is None else t_hi
    if out is None:
        out = torch.empty((t_hi - t_lo + 1, W), dtype=acc, device=img.device)
    out_code, out_pitch = _dev2d(out, "out")
    _shape(out, (t_hi - t_lo + 1, W), "out")
    ws = _workspace(workspace, workspace_size_sheared(h, w, q, img.dtype, out.dtype),
                    img.device)
    _check(lib.fht_forward_sheared(_ptr(img), in_code, h, w, in_pitch, q, float(spl), t_lo,
                                   t_hi, _ptr(out), out_code, out_pitch, _ptr(ws), _nbytes(ws),
                                   _stream(stream)), "fht_forward_sheared")
    return out


# ------------------------------------------------------------------ scaled (Section 4)

def scaled_width(w: int, alpha: float) -> int:
    """Columns of a row of w pixels scaled by alpha (fht_scaled_width)."""
    wa = ctypes.c_int()
    _check(lib.fht_scaled_width(w, float(alpha), ctypes.byref(wa)), "fht_scaled_width")
    return wa.value


def scaled_shape(h: int, w: int, q: int, alpha: float) -> tuple[int, int]:
    """(n, W) of the scaled quadrant q of an h x w image (fht_scaled_shape)."""
    r, c = ctypes.c_int(), ctypes.c_int()
    _check(lib.fht_scaled_shape(h, w, q, float(alpha), ctypes.byref(r), ctypes.byref(c)),
           "fht_scaled_shape")
    return r.value, c.value


def workspace_size_scaled(h: int, w: int, q: int, alpha: float, in_dtype: torch.dtype,
                          acc: torch.dtype) -> int:
    n = ctypes.c_size_t()
    _check(lib.fht_workspace_size_scaled(h, w, q, float(alpha), _DTYPE[in_dtype], _DTYPE[acc],
                                         ctypes.byref(n)), "fht_workspace_size_scaled")
    return n.value


def scale_range(phi_lo: float, phi_hi: float, h: int,
                w: int) -> tuple[int, float, float, int, int]:
    """(q, alpha, spl, t_lo, t_hi): the one scaled and sheared quadrant and
    its slope rows for the line angles [phi_lo, phi_hi] degrees
    (fht_scale_range)."""
    q, t_lo, t_hi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    alpha, spl = ctypes.c_double(), ctypes.c_double()
    _check(lib.fht_scale_range(phi_lo, phi_hi, h, w, ctypes.byref(q), ctypes.byref(alpha),
                               ctypes.byref(spl), ctypes.byref(t_lo), ctypes.byref(t_hi)),
           "fht_scale_range")
    return q.value, alpha.value, spl.value, t_lo.value, t_hi.value


def forward_scaled(img: torch.Tensor, q: int, alpha: float, spl: float = 0.0, t_lo: int = 0,
                   t_hi: int | None = None, acc: torch.dtype = torch.int32,
                   out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Rows t_lo..t_hi of quadrant q of the image scaled along its rows by
    alpha, then sheared by spl per row (Section 4; fht_forward_scaled)."""
    in_code, in_pitch = _dev2d(img, "img")
    h, w = img.shape
    n, W = scaled_shape(h, w, q, alpha)
    t_hi = n - 1 if t_hi is None else t_hi
    if out is None:
        out = torch.empty((t_hi - t_lo + 1, W), dtype=acc, device=img.device)
    out_code, out_pitch = _dev2d(out, "out")
    _shape(out, (t_hi - t_lo + 1, W), "out")
    ws = _workspace(workspace, workspace_size_scaled(h, w, q, alpha, img.dtype, out.dtype),
                    img.device)
    _check(lib.fht_forward_scaled(_ptr(img), in_code, h, w, in_pitch, q, float(alpha),
                                  float(spl), t_lo, t_hi, _ptr(out), out_code, out_pitch,
                                  _ptr(ws), _nbytes(ws), _stream(stream)),
           "fht_forward_scaled")
    return out


# ------------------------------------------------------------------ strips of one image

def workspace_size_padded(h: int, w: int, q: int, n: int, W: int, in_dtype: torch.dtype,
                          acc: torch.dtype) -> int:
    b = ctypes.c_size_t()
    _check(lib.fht_workspace_size_padded(h, w, q, n, W, _DTYPE[in_dtype], _DTYPE[acc],
                                         ctypes.byref(b)), "fht_workspace_size_padded")
    return b.value


def forward_padded(img: torch.Tensor, q: int, n: int, W: int, acc: torch.dtype = torch.int32,
                   out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Quadrant q of img zero-padded to n rows (of the transposed image for
    Q2/Q3) on the cyclic width W: (n, W) (fht_forward_padded). img may have
    no rows (an empty strip)."""
    h, w = img.shape
    if out is None:
        out = torch.empty((n, W), dtype=acc, device=img.device)
    out_code, out_pitch = _dev2d(out, "out")
    _shape(out, (n, W), "out")
    if img.numel() == 0:
        _check(lib.fht_forward_padded(None, _DTYPE[img.dtype], h, w, max(w, 1), q, n, W,
                                      _ptr(out), out_code, out_pitch, None, 0, _stream(stream)),
               "fht_forward_padded")
        return out
    in_code, in_pitch = _dev2d(img, "img")
    ws = _workspace(workspace, workspace_size_padded(h, w, q, n, W, img.dtype, out.dtype),
                    img.device)
    _check(lib.fht_forward_padded(_ptr(img), in_code, h, w, in_pitch, q, n, W, _ptr(out),
                                  out_code, out_pitch, _ptr(ws), _nbytes(ws), _stream(stream)),
           "fht_forward_padded")
    return out


def merge_strips(parts: torch.Tensor, q: int, tau0: int, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """The last log2(P) levels of a sharded quadrant (fht_merge_strips):
    parts (P, rows, W) holds every strip's level rows tau0 .. tau0+rows-1;
    returns (rows*P, W), row (tau - tau0)*P + c = final slope tau*P + c."""
    P, rows, W = parts.shape
    if parts.dtype not in (torch.int32, torch.float32) or not parts.is_cuda:
        raise ValueError("parts: int32 or float32 CUDA tensor")
    if parts.stride(2) != 1:
        raise ValueError("parts: unit column stride")
    if out is None:
        out = torch.empty((rows * P, W), dtype=parts.dtype, device=parts.device)
    out_code, out_pitch = _dev2d(out, "out")
    _shape(out, (rows * P, W), "out")
    if out.dtype != parts.dtype:
        raise ValueError("out: same dtype as parts")
    _check(lib.fht_merge_strips(_ptr(parts), _DTYPE[parts.dtype], P, rows, W,
                                parts.stride(0), parts.stride(1), tau0, q, _ptr(out),
                                out_pitch, _stream(stream)), "fht_merge_strips")
    return out


class BatchPlan:
    """Many images of different sizes, each transformed as `forward` would
    (one quadrant, one type pair), in one persistent launch; float32 plans
    also run the batch's adjoint (`adjoint`) the same way."""

    def __init__(self, shapes, q: int = Q0, in_dtype: torch.dtype = torch.uint8,
                 acc: torch.dtype = torch.int32):
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        self.q, self.in_dtype, self.acc = q, in_dtype, acc
        n = len(self.shapes)
        hs = (ctypes.c_int * n)(*[h for h, _ in self.shapes])
        ws = (ctypes.c_int * n)(*[w for _, w in self.shapes])
        plan = ctypes.c_void_p()
        nbytes = ctypes.c_size_t()
        _check(lib.fht_plan_create_batched(hs, ws, n, q, _DTYPE[in_dtype], _DTYPE[acc],
                                           ctypes.byref(plan), ctypes.byref(nbytes)),
               "fht_plan_create_batched")
        self._plan = plan
        self.workspace_bytes = nbytes.value
        self.out_shapes = [query_shape(h, w, q) for h, w in self.shapes]
        self._in_sizes = [torch.Size(sh) for sh in self.shapes]
        self._out_sizes = [torch.Size(sh) for sh in self.out_shapes]

    def _reject(self, j, x, o):
        """Raise the precise error for image j / output j."""
        _dev2d(x, "img")
        _dev2d(o, "out")
        if tuple(x.shape) != self.shapes[j] or x.dtype != self.in_dtype:
            raise ValueError(f"image {j}: expected {self.shapes[j]} {self.in_dtype}")
        _shape(o, self.out_shapes[j], f"out[{j}]")
        if o.dtype != self.acc:
            raise ValueError(f"out[{j}] must be {self.acc}")
        raise ValueError(f"image {j} or out[{j}] is not a usable 2-D CUDA tensor")

    def workspace(self, device) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=device)

    def forward(self, imgs, outs=None, workspace: torch.Tensor | None = None,
                stream=None):
        if len(imgs) != len(self.shapes):
            raise ValueError("one image per planned shape")
        dev = imgs[0].device
        if outs is None:
            outs = [torch.empty(sh, dtype=self.acc, device=dev) for sh in self.out_shapes]
        rows = []
        for j, (x, o) in enumerate(zip(imgs, outs)):
            xs, os_ = x.stride(), o.stride()
            if (x.dtype != self.in_dtype or o.dtype != self.acc or not x.is_cuda
                    or not o.is_cuda or x.shape != self._in_sizes[j]
                    or o.shape != self._out_sizes[j] or xs[1] != 1 or os_[1] != 1):
                self._reject(j, x, o)
            rows.append((x.data_ptr(), max(xs[0], x.shape[1]),
                         o.data_ptr(), max(os_[0], o.shape[1])))
        # fht_image_desc is {img, img_pitch, out, out_pitch}, 8 bytes each
        descs = np.array(rows, dtype=np.int64)
        ws = self.workspace(dev) if workspace is None else workspace
        if ws.numel() * ws.element_size() < self.workspace_bytes:
            raise ValueError("workspace too small")
        _check(lib.fht_forward_batched(self._plan, ctypes.c_void_p(descs.ctypes.data),
                                       _ptr(ws), _nbytes(ws), _stream(stream)),
               "fht_forward_batched")
        self._last_ws = ws
        return outs

    def adjoint(self, grads, outs=None, workspace: torch.Tensor | None = None,
                stream=None):
        """Image gradients of the batch (float32 plans): outs[j] = H_j^T
        grads[j], each as `adjoint(grads[j], h_j, w_j, LAYOUT_QUADRANT, q)`
        would compute it, in one persistent launch."""
        if self.acc != torch.float32:
            raise ValueError("the batched adjoint needs a float32 plan")
        if len(grads) != len(self.shapes):
            raise ValueError("one gradient per planned shape")
        dev = grads[0].device
        if outs is None:
            outs = [torch.empty(sh, dtype=torch.float32, device=dev) for sh in self.shapes]
        rows = []
        for j, (g, o) in enumerate(zip(grads, outs)):
            for t, name, want in ((g, f"grads[{j}]", self._out_sizes[j]),
                                  (o, f"outs[{j}]", self._in_sizes[j])):
                _dev2d(t, name)
                if t.dtype != torch.float32:
                    raise ValueError(f"{name} must be float32")
                if t.shape != want:
                    raise ValueError(f"{name}: expected shape {tuple(want)}")
            rows.append((g.data_ptr(), max(g.stride(0), g.shape[1]),
                         o.data_ptr(), max(o.stride(0), o.shape[1])))
        # fht_adjoint_desc is {grad_hough, pitch, grad_img, pitch}, 8 bytes each
        descs = np.array(rows, dtype=np.int64)
        ws = self.workspace(dev) if workspace is None else workspace
        if ws.numel() * ws.element_size() < self.workspace_bytes:
            raise ValueError("workspace too small")
        _check(lib.fht_adjoint_batched(self._plan, ctypes.c_void_p(descs.ctypes.data),
                                       _ptr(ws), _nbytes(ws), _stream(stream)),
               "fht_adjoint_batched")
        self._last_ws = ws
        return outs

    def status(self, workspace: torch.Tensor | None = None, stream=None) -> int:
        """Device status of the last launch on `workspace` (0 = ok, 5 = a
        dependency wait timed out); waits for the stream."""
        ws = self._last_ws if workspace is None else workspace
        return int(lib.fht_batched_status(self._plan, _ptr(ws), _stream(stream)))

    def set_test_hooks(self, wait_budget_cycles: int, dep_bias: int) -> None:
        _check(lib.fht_batched_test_hooks(self._plan, wait_budget_cycles, dep_bias),
               "fht_batched_test_hooks")

    def __del__(self):
        plan = getattr(self, "_plan", None)
        if plan is not None and plan.value:
            lib.fht_plan_destroy(plan)
            self._plan = None


# ------------------------------------------------------------------ profiling

class _KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_int),
                ("total_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double)]


def profile_begin() -> None:
    """Bracket every following library launch with CUDA events on its stream."""
    _check(lib.fht_profile_begin(), "fht_profile_begin")


def profile_end() -> dict[str, tuple[int, float, float]]:
    """Stop recording; {kernel name: (launches, summed device ms, summed
    algorithmic bytes)}."""
    cap = 64
    arr = (_KernelTime * cap)()
    cnt = ctypes.c_int()
    _check(lib.fht_profile_end(ctypes.cast(arr, ctypes.c_void_p), cap, ctypes.byref(cnt)),
           "fht_profile_end")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms, arr[i].alg_bytes)
            for i in range(min(cnt.value, cap))}


def launch_count() -> int:
    """Kernel launches issued by the library since it was loaded."""
    return int(lib.fht_launch_count())


def device_status() -> int:
    """Wait for the device; FHT_EBOUNDS if a kernel of the debug build
    refused an access outside its pass's buffers since the last call (the
    count is reset), else FHT_OK."""
    return int(lib.fht_device_status())


# ------------------------------------------------------------ uniform batches

def _dev3d(t: torch.Tensor, name: str) -> tuple[int, int]:
    """(pitch, batch stride) in elements of a float32 (B, rows, cols) CUDA tensor."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise ValueError(f"{name} must be a float32 CUDA tensor")
    if t.dim() != 3 or t.stride(2) != 1:
        raise ValueError(f"{name} must be 3-D (batch, rows, cols) with unit column stride")
    return max(t.stride(1), t.shape[2]), t.stride(0)


def workspace_size_many(batch: int, h: int, w: int, layout: int = LAYOUT_FULL,
                        q: int = Q0) -> int:
    """Workspace bytes of forward_many / adjoint_many on `batch` h x w images."""
    n = ctypes.c_size_t()
    _check(lib.fht_workspace_size_many(batch, h, w, layout, q, ctypes.byref(n)),
           "fht_workspace_size_many")
    return n.value


def forward_many(imgs: torch.Tensor, layout: int = LAYOUT_FULL, q: int = Q0,
                 out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """FP32 transforms of a (B, h, w) batch of same-size images in one launch
    per pass: (B, rows, cols), each as full_quadrants (layout FULL) or
    forward of quadrant q (layout QUADRANT)."""
    ip, ib = _dev3d(imgs, "imgs")
    B, h, w = imgs.shape
    rows, cols = full_shape(h, w) if layout == LAYOUT_FULL else query_shape(h, w, q)
    if out is None:
        out = torch.empty((B, rows, cols), dtype=torch.float32, device=imgs.device)
    _shape(out, (B, rows, cols), "out")
    op, ob = _dev3d(out, "out")
    ws = _workspace(workspace, workspace_size_many(B, h, w, layout, q), imgs.device)
    _check(lib.fht_forward_many(_ptr(imgs), B, ib, h, w, ip, layout, q, _ptr(out), ob, op,
                                _ptr(ws), _nbytes(ws), _stream(stream)), "fht_forward_many")
    return out


def adjoint_many(grads: torch.Tensor, h: int, w: int, layout: int = LAYOUT_FULL, q: int = Q0,
                 out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """Adjoints of a (B, rows, cols) batch of FP32 Hough-image gradients in
    one launch per pass: (B, h, w)."""
    gp, gb = _dev3d(grads, "grads")
    B = grads.shape[0]
    rows, cols = full_shape(h, w) if layout == LAYOUT_FULL else query_shape(h, w, q)
    _shape(grads, (B, rows, cols), "grads")
    if out is None:
        out = torch.empty((B, h, w), dtype=torch.float32, device=grads.device)
    _shape(out, (B, h, w), "out")
    op, ob = _dev3d(out, "out")
    ws = _workspace(workspace, workspace_size_many(B, h, w, layout, q), grads.device)
    _check(lib.fht_adjoint_many(_ptr(grads), B, gb, h, w, layout, q, gp, _ptr(out), ob, op,
                                _ptr(ws), _nbytes(ws), _stream(stream)), "fht_adjoint_many")
    return out


class FHTFunction(torch.autograd.Function):
    """Differentiable FP32 Hough transform: forward by the CUDA butterfly,
    backward by the hand-written adjoint kernels (its exact transpose).

    apply(x, layout=LAYOUT_FULL, q=Q0) for a float32 CUDA tensor x of shape
    (h, w), or (B, h, w) for a batch of same-size images (one launch per pass
    for the whole batch)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, layout: int = LAYOUT_FULL, q: int = Q0):
        ctx.h, ctx.w = x.shape[-2:]
        ctx.layout, ctx.q = layout, q
        x = x.contiguous()

        def one(img):
            if layout == LAYOUT_FULL:
                return full_quadrants(img, acc=torch.float32)
            return forward(img, q, acc=torch.float32)

        if x.dim() == 2:
            return one(x)
        return forward_many(x, layout, q)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        g = g.contiguous()
        if g.dim() == 2:
            return adjoint(g, ctx.h, ctx.w, ctx.layout, ctx.q), None, None
        return adjoint_many(g, ctx.h, ctx.w, ctx.layout, ctx.q), None, None


_load_default_tuning()
