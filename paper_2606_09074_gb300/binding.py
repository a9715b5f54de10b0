"""Python binding of librefine, the GB300 (sm_103a) implementation of REFINE's
rendering-free primitive importance, ratio pruning and compaction
(arXiv 2606.09074, Sec. 3.2-3.3).

The functions named ``refine_*`` mirror the C ABI in ``include/refine.h``
one to one (ctypes, argument marshalling only).  ``Context`` wraps them for
PyTorch tensors: PyTorch supplies device memory and streams; every step of
the computation runs in librefine's CUDA kernels.  There is no CPU path: if
the shared library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build
from .synth import CAMERA_DTYPE

LIB_PATH = _build.LIB

REFINE_OK = 0
REFINE_EINVAL = 1
REFINE_ENOMEM = 2
REFINE_ECUDA = 3
REFINE_ENONFINITE = 4
REFINE_ETIMEOUT = 5
REFINE_EBUSY = 6
REFINE_ECANCELLED = 7
REFINE_ENOTFOUND = 8
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ETIMEOUT",
                6: "EBUSY", 7: "ECANCELLED", 8: "ENOTFOUND"}

REFINE_F32 = 0
TIMING_ALL = 1    # REFINE_TIMING_ALL
TIMING_SCORE = 2  # REFINE_TIMING_SCORE
REFINE_BF16 = 1
REFINE_BF16S = 2  # log-scale rows float32, the other 53 rows bfloat16

FLAG_NO_VIS = 1 << 0
FLAG_NO_PROJ = 1 << 1
FLAG_EQUAL_LAMBDA = 1 << 2
FLAG_NORM_ATTR = 1 << 3
FLAG_FULL_JACOBIAN = 1 << 4


class RefineError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class refine_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("zfar", C.c_float)]


class refine_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("dtype", C.c_int32), ("reserved", C.c_int32),
                ("pos", C.c_void_p), ("attr", C.c_void_p), ("row_stride", C.c_int64)]


class refine_params(C.Structure):
    _fields_ = [("eta", C.c_float), ("luma", C.c_float * 3), ("e_ln_gem", C.c_double),
                ("e_col", C.c_double), ("e_opa", C.c_double), ("flags", C.c_int32),
                ("max_views", C.c_int32)]


_WORK_COUNTERS = ("visible_mixed_pairs", "open_u_pairs", "open_v_pairs", "open_z_pairs", "bound_u_pairs",
                  "bound_v_pairs", "exact_u_pairs", "exact_v_pairs", "exact_warp_axes")


class refine_scene_stats(C.Structure):
    _fields_ = [("F_col", C.c_double), ("F_opa", C.c_double), ("F_gem", C.c_double),
                ("lambda_t", C.c_double * 3), ("lambda_", C.c_double * 3), ("mean_m", C.c_double * 3),
                ("pairs", C.c_int64), ("tile_views", C.c_int64), ("in_pairs", C.c_int64),
                ("out_pairs", C.c_int64), ("mixed_pairs", C.c_int64), ("bound_pairs", C.c_int64),
                ("footprint_pairs", C.c_int64)] + [(k, C.c_int64) for k in _WORK_COUNTERS]

    def as_dict(self):
        d = {"F_col": self.F_col, "F_opa": self.F_opa, "F_gem": self.F_gem,
             "lambda_t": list(self.lambda_t), "lambda": list(self.lambda_),
             "mean_m": list(self.mean_m), "pairs": self.pairs, "tile_views": self.tile_views,
             "in_pairs": self.in_pairs, "out_pairs": self.out_pairs, "mixed_pairs": self.mixed_pairs,
             "bound_pairs": self.bound_pairs, "footprint_pairs": self.footprint_pairs}
        d.update({k: getattr(self, k) for k in _WORK_COUNTERS})
        return d


class refine_job(C.Structure):
    _fields_ = [("scene", refine_scene), ("cams_dev", C.c_void_p), ("n_views", C.c_int32),
                ("reserved", C.c_int32), ("ratio", C.c_double), ("scores_dev", C.c_void_p),
                ("keep_mask_dev", C.c_void_p), ("out_pos_dev", C.c_void_p), ("out_attr_dev", C.c_void_p),
                ("out_row_stride", C.c_int64), ("kept_idx_dev", C.c_void_p)]


class refine_shape(C.Structure):
    _fields_ = [("tile", C.c_int32), ("cta_threads", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("camera_block", C.c_int32), ("ms", C.c_double)]


class refine_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("dtype", C.c_int32), ("n_views", C.c_int32), ("pos_host", C.c_void_p),
                ("attr_host", C.c_void_p), ("cams_host", C.c_void_p), ("ratio", C.c_double),
                ("params", C.c_void_p), ("keep_mask_host", C.c_void_p), ("scores_host", C.c_void_p),
                ("out_pos_host", C.c_void_p), ("out_attr_host", C.c_void_p), ("kept_idx_host", C.c_void_p)]


class refine_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("round_size", C.c_int32), ("n_keep", C.c_int64),
                ("threshold", C.c_float), ("reserved", C.c_float), ("submit_ms", C.c_double),
                ("admit_ms", C.c_double), ("done_ms", C.c_double), ("copied_ms", C.c_double),
                ("prepped_ms", C.c_double), ("scored_ms", C.c_double), ("computed_ms", C.c_double),
                ("read_ms", C.c_double)]


class refine_queue_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rounds", C.c_int64), ("pending", C.c_int64), ("in_flight", C.c_int64),
                ("bytes_in_use", C.c_uint64), ("peak_bytes", C.c_uint64), ("budget_bytes", C.c_uint64),
                ("max_round", C.c_int32), ("slots", C.c_int32), ("kernel_launches", C.c_int64),
                ("dispatch_ms", C.c_double), ("retire_ms", C.c_double)]


assert C.sizeof(refine_camera) == 80 and C.sizeof(refine_scene) == 40 and C.sizeof(refine_job) == 112
assert C.sizeof(refine_params) == 48
assert C.sizeof(refine_shape) == 24
assert C.sizeof(refine_request) == 96 and C.sizeof(refine_result) == 88 and C.sizeof(refine_queue_stats) == 104

_P = C.c_void_p
_SIGNATURES = {
    "refine_version": (C.c_char_p, []),
    "refine_params_default": (C.c_int, [C.POINTER(refine_params)]),
    "refine_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "refine_ctx_destroy": (None, [_P]),
    "refine_last_error": (C.c_char_p, [_P]),
    "refine_score": (C.c_int, [_P, C.POINTER(refine_scene), _P, C.c_int32, C.POINTER(refine_params),
                               _P, _P]),
    "refine_score_ex": (C.c_int, [_P, C.POINTER(refine_scene), _P, C.c_int32,
                                  C.POINTER(refine_params), _P, _P, C.POINTER(refine_scene_stats), _P]),
    "refine_select": (C.c_int, [_P, _P, C.c_int64, C.c_double, _P, C.POINTER(C.c_float),
                                C.POINTER(C.c_int64), _P]),
    "refine_compact": (C.c_int, [_P, C.POINTER(refine_scene), _P, _P, _P, C.c_int64, _P,
                                 C.POINTER(C.c_int64), _P]),
    "refine_prune_host": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P, C.c_int32,
                                    C.POINTER(refine_params), C.c_double, _P, _P, _P, _P,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_float), _P]),
    "refine_select_noalloc": (C.c_int, [_P, C.c_int64, C.c_double, _P, C.POINTER(C.c_float),
                                        C.POINTER(C.c_int64), C.c_char_p, C.c_size_t, _P]),
    "refine_batch_create": (C.c_int, [_P, C.POINTER(refine_job), C.c_int32, C.POINTER(refine_params),
                                      C.POINTER(C.c_void_p)]),
    "refine_batch_run": (C.c_int, [_P, _P]),
    "refine_batch_results": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_float), _P]),
    "refine_batch_launches": (C.c_int64, [_P]),
    "refine_batch_destroy": (None, [_P]),
    "refine_autotune": (C.c_int, [_P, C.POINTER(refine_job), C.c_int32, C.POINTER(refine_params), C.c_int32,
                                  C.POINTER(refine_shape), C.POINTER(refine_shape), C.c_int32,
                                  C.POINTER(C.c_int32)]),
    "refine_ctx_get_shape": (C.c_int, [_P, C.POINTER(refine_shape)]),
    "refine_ctx_set_shape": (C.c_int, [_P, C.POINTER(refine_shape)]),
    "refine_queue_footprint": (C.c_uint64, [C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_int32]),
    "refine_queue_create": (C.c_int, [_P, C.c_uint64, C.c_int32, C.POINTER(refine_params),
                                      C.POINTER(C.c_void_p)]),
    "refine_queue_submit": (C.c_int, [_P, C.POINTER(refine_request), C.POINTER(C.c_uint64)]),
    "refine_queue_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(refine_result), C.c_int32]),
    "refine_queue_poll_any": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(refine_result), C.c_int32]),
    "refine_queue_stats_get": (C.c_int, [_P, C.POINTER(refine_queue_stats)]),
    "refine_queue_destroy": (None, [_P]),
    "refine_queue_last_error": (C.c_char_p, [_P]),
    "refine_write_ply": (C.c_int, [C.c_char_p, C.c_int64, C.c_int32, _P, _P, C.c_int64]),
    "refine_read_ply": (C.c_int, [C.c_char_p, C.POINTER(C.c_int64), _P, _P, C.c_int64]),
    "refine_ctx_check": (C.c_int, [_P, _P]),
    "refine_ctx_set_timing": (C.c_int, [_P, C.c_int]),
    "refine_ctx_kernel_times": (C.c_int, [_P, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int64), C.c_int32, C.POINTER(C.c_int32)]),
    "refine_ctx_launch_count": (C.c_int64, [_P]),
    "refine_selftest_wait": (C.c_int, [_P, C.c_uint32, C.c_uint32, C.c_int64, _P]),
    "refine_fma_rate": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), _P]),
}


def _load():
    import torch  # noqa: F401  -- loads the CUDA runtime that librefine shares with PyTorch
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"librefine is not built ({LIB_PATH} is missing). Build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` or "
            "`python paper_2606_09074_gb300/build.py`. There is no CPU fallback.")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
globals().update({name: getattr(_lib, name) for name in _SIGNATURES})


def library_path() -> str:
    return LIB_PATH


def default_params(**overrides) -> refine_params:
    p = refine_params()
    refine_params_default(C.byref(p))  # noqa: F821
    for k, v in overrides.items():
        if k == "luma":
            p.luma[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def _check(ctx, st):
    if st != REFINE_OK:
        raise RefineError(st, refine_last_error(ctx).decode(errors="replace"))  # noqa: F821


def _stream_handle(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return C.c_void_p(stream.cuda_stream)


class MixedRows:
    """The 56 attribute rows of a scene in the REFINE_BF16S layout, in one
    byte buffer: the 3 log-scale rows float32 ([3, stride]), then the other 53
    rows bfloat16 ([53, stride]).  It stands where the float32 or bfloat16
    [56, n] tensor stands elsewhere in this binding: ``shape``, ``stride``,
    ``data_ptr``, ``[:, :k]`` column views, ``to``/``cpu``, ``is_pinned``."""

    dtype = "bf16s"
    NF = 3

    def __init__(self, buf, n: int, stride: int):
        self.buf, self.n, self.row_stride = buf, int(n), int(stride)

    @classmethod
    def empty(cls, n: int, stride: int | None = None, device=None, pin_memory: bool = False):
        import torch
        stride = max(int(n), 1) if stride is None else int(stride)
        buf = torch.empty(stride * (4 * cls.NF + 2 * (56 - cls.NF)), dtype=torch.uint8, device=device,
                          pin_memory=pin_memory)
        return cls(buf, n, stride)

    @classmethod
    def from_float(cls, attr, device=None, pin_memory: bool = False):
        """Rows of a float32 [56, n] array or tensor, the last 53 rounded to
        bfloat16 (round to nearest even)."""
        import torch
        a = torch.as_tensor(attr, dtype=torch.float32)
        out = cls.empty(a.shape[1], device=device, pin_memory=pin_memory)
        out.f32_rows()[:, : out.n].copy_(a[: cls.NF])
        out.bf16_rows()[:, : out.n].copy_(a[cls.NF:].to(torch.bfloat16))
        return out

    def f32_rows(self):
        import torch
        return self.buf[: 4 * self.NF * self.row_stride].view(torch.float32).view(self.NF, self.row_stride)

    def bf16_rows(self):
        import torch
        o = 4 * self.NF * self.row_stride
        return self.buf[o: o + 2 * (56 - self.NF) * self.row_stride].view(torch.bfloat16).view(
            56 - self.NF, self.row_stride)

    def float(self):
        """The rows widened to a float32 [56, n] tensor (exact)."""
        import torch
        return torch.cat([self.f32_rows()[:, : self.n], self.bf16_rows()[:, : self.n].float()], 0)

    @property
    def shape(self):
        return (56, self.n)

    @property
    def device(self):
        return self.buf.device

    def stride(self, dim: int) -> int:
        return self.row_stride if dim == 0 else 1

    def data_ptr(self) -> int:
        return self.buf.data_ptr()

    def is_pinned(self) -> bool:
        return self.buf.is_pinned()

    def to(self, device, non_blocking: bool = False):
        return MixedRows(self.buf.to(device, non_blocking=non_blocking), self.n, self.row_stride)

    def cpu(self):
        return self.to("cpu")

    def pin_memory(self):
        return MixedRows(self.buf.pin_memory(), self.n, self.row_stride)

    col_bytes = 4 * NF + 2 * (56 - NF)  # bytes of the 56 rows per element of the stride

    def __getitem__(self, key):
        rows, cols = key
        if rows != slice(None) or not isinstance(cols, slice) or cols.start not in (None, 0) or cols.step not in (None, 1):
            raise IndexError("MixedRows supports [:, :k] column views only")
        k = self.n if cols.stop is None else min(int(cols.stop), self.n)
        return MixedRows(self.buf, k, self.row_stride)


def empty_attr_like(attr, cols: int, device=None, pin_memory: bool = False):
    """An uninitialised [56, cols] attribute block of the same storage type
    as ``attr`` (a float32 or bfloat16 tensor, or MixedRows)."""
    import torch
    if isinstance(attr, MixedRows):
        return MixedRows.empty(cols, device=device, pin_memory=pin_memory)
    return torch.empty((56, cols), dtype=attr.dtype, device=device, pin_memory=pin_memory)


def attr_col_bytes(attr) -> int:
    """Bytes of the 56 attribute rows per primitive: 224 (float32), 112
    (bfloat16) or 118 (MixedRows)."""
    return MixedRows.col_bytes if isinstance(attr, MixedRows) else 56 * attr.element_size()


def _dtype_code(t) -> int:
    import torch
    if isinstance(t, MixedRows):
        return REFINE_BF16S
    if t.dtype == torch.float32:
        return REFINE_F32
    if t.dtype in (torch.bfloat16, torch.int16, torch.uint16):
        return REFINE_BF16
    raise TypeError(f"unsupported attribute dtype {t.dtype}")


def make_scene(pos, attr) -> refine_scene:
    """refine_scene view of device tensors pos [3, n] float32 and attr
    [56, n] float32 / bfloat16 with a common row stride."""
    n = pos.shape[1]
    if pos.shape[0] != 3 or attr.shape[0] != 56 or attr.shape[1] != n:
        raise ValueError("expected pos [3, n] and attr [56, n]")
    if n and (pos.stride(1) != 1 or attr.stride(1) != 1 or pos.stride(0) != attr.stride(0)):
        raise ValueError("pos and attr must be row-contiguous with the same row stride")
    sc = refine_scene()
    sc.n = n
    sc.dtype = _dtype_code(attr)
    sc.pos = pos.data_ptr()
    sc.attr = attr.data_ptr()
    sc.row_stride = pos.stride(0) if n else 0
    return sc


def cameras_to_device(cams, device):
    """Uploads a ``synth.CAMERA_DTYPE`` array as raw refine_camera records."""
    import torch
    arr = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
    return torch.from_numpy(arr.view(np.uint8).copy()).to(device)


class Context:
    """A librefine context bound to one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        st = refine_ctx_create(C.byref(h), device)  # noqa: F821
        if st != REFINE_OK:
            raise RefineError(st, f"refine_ctx_create(device={device}) failed")
        self.handle = h

    def close(self):
        if self.handle:
            refine_ctx_destroy(self.handle)  # noqa: F821
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------
    def score(self, pos, attr, cams_dev, n_views=None, params=None, scores=None, view_sum=None,
              stats=False, stream=None):
        """Importance scores (float32 [n]).  ``cams_dev`` is a device uint8
        tensor of refine_camera records.  With ``stats`` also returns the
        scene statistics dict (synchronises)."""
        import torch
        sc = make_scene(pos, attr)
        V = n_views if n_views is not None else cams_dev.numel() // 80
        if scores is None:
            scores = torch.empty(sc.n, dtype=torch.float32, device=self.device)
        st_out = refine_scene_stats() if stats else None
        rc = refine_score_ex(self.handle, C.byref(sc), C.c_void_p(cams_dev.data_ptr()), V,  # noqa: F821
                             C.byref(params) if params is not None else None,
                             C.c_void_p(scores.data_ptr()),
                             C.c_void_p(view_sum.data_ptr()) if view_sum is not None else None,
                             C.byref(st_out) if stats else None, _stream_handle(stream, self.device))
        _check(self.handle, rc)
        return (scores, st_out.as_dict()) if stats else scores

    def select(self, scores, ratio, mask=None, threshold=True, stream=None):
        """Returns (keep mask uint32 words as int32 tensor, threshold or None, n_keep)."""
        import torch
        n = scores.numel()
        if mask is None:
            mask = torch.empty(max((n + 31) // 32, 1), dtype=torch.int32, device=self.device)
        thr = C.c_float()
        nk = C.c_int64()
        rc = refine_select(self.handle, C.c_void_p(scores.data_ptr()), n, float(ratio),  # noqa: F821
                           C.c_void_p(mask.data_ptr()), C.byref(thr) if threshold else None,
                           C.byref(nk), _stream_handle(stream, self.device))
        _check(self.handle, rc)
        return mask, (thr.value if threshold else None), nk.value

    def compact(self, pos, attr, mask, n_keep, out_pos=None, out_attr=None, kept_idx=True,
                out_row_stride=None, return_count=False, stream=None):
        """Compacts the kept primitives; returns (out_pos, out_attr, kept_idx[, count])."""
        import torch
        sc = make_scene(pos, attr)
        stride = out_row_stride if out_row_stride is not None else max(n_keep, 1)
        if out_pos is None:
            out_pos = torch.empty((3, stride), dtype=torch.float32, device=self.device)
        if out_attr is None:
            out_attr = empty_attr_like(attr, stride, device=self.device)
        idx = torch.empty(max(n_keep, 1), dtype=torch.int32, device=self.device) if kept_idx else None
        cnt = C.c_int64()
        rc = refine_compact(self.handle, C.byref(sc), C.c_void_p(mask.data_ptr()),  # noqa: F821
                            C.c_void_p(out_pos.data_ptr()), C.c_void_p(out_attr.data_ptr()), stride,
                            C.c_void_p(idx.data_ptr()) if idx is not None else None,
                            C.byref(cnt) if return_count else None, _stream_handle(stream, self.device))
        _check(self.handle, rc)
        out = (out_pos[:, :n_keep], out_attr[:, :n_keep], idx[:n_keep] if idx is not None else None)
        return out + (cnt.value,) if return_count else out

    def prune_host(self, pos_host, attr_host, cams, ratio, params=None, want_scores=False,
                   out=None, stream=None):
        """Whole pass from host tensors (ideally pinned).  Returns a dict with
        out_pos, out_attr, idx, (scores), n_keep, threshold."""
        import torch
        n = pos_host.shape[1]
        dt = _dtype_code(attr_host)
        cams_arr = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        n_keep = n - int(np.floor(float(ratio) * n))
        if out is None:
            pin = pos_host.is_pinned()
            out = {"out_pos": torch.empty((3, max(n_keep, 1)), dtype=torch.float32, pin_memory=pin),
                   "out_attr": empty_attr_like(attr_host, max(n_keep, 1), pin_memory=pin),
                   "idx": torch.empty(max(n_keep, 1), dtype=torch.int32, pin_memory=pin)}
            if want_scores:
                out["scores"] = torch.empty(max(n, 1), dtype=torch.float32, pin_memory=pin)
        nk = C.c_int64()
        thr = C.c_float()
        rc = refine_prune_host(self.handle, n, dt, C.c_void_p(pos_host.data_ptr()),  # noqa: F821
                               C.c_void_p(attr_host.data_ptr()),
                               cams_arr.ctypes.data_as(C.c_void_p), len(cams_arr),
                               C.byref(params) if params is not None else None, float(ratio),
                               C.c_void_p(out["out_pos"].data_ptr()),
                               C.c_void_p(out["out_attr"].data_ptr()),
                               C.c_void_p(out["idx"].data_ptr()),
                               C.c_void_p(out["scores"].data_ptr()) if "scores" in out else None,
                               C.byref(nk), C.byref(thr), _stream_handle(stream, self.device))
        _check(self.handle, rc)
        res = {"out_pos": out["out_pos"][:, :nk.value], "out_attr": out["out_attr"][:, :nk.value],
               "idx": out["idx"][:nk.value], "n_keep": nk.value, "threshold": thr.value}
        if "scores" in out:
            res["scores"] = out["scores"][:n]
        return res

    def check(self, stream=None):
        _check(self.handle, refine_ctx_check(self.handle, _stream_handle(stream, self.device)))  # noqa: F821

    def status(self, stream=None) -> int:
        return refine_ctx_check(self.handle, _stream_handle(stream, self.device))  # noqa: F821

    def set_timing(self, on, score_only: bool = False):
        """Brackets kernel launches with CUDA events: every launch, or only
        the score kernel's (score_only: two events per pass)."""
        mode = 0 if not on else (TIMING_SCORE if score_only else TIMING_ALL)
        _check(self.handle, refine_ctx_set_timing(self.handle, mode))  # noqa: F821

    def kernel_times(self) -> dict:
        cap = 32
        names = (C.c_char_p * cap)()
        ms = (C.c_double * cap)()
        ln = (C.c_int64 * cap)()
        cnt = C.c_int32()
        _check(self.handle, refine_ctx_kernel_times(self.handle, names, ms, ln, cap, C.byref(cnt)))  # noqa: F821
        return {names[i].decode(): {"ms": ms[i], "launches": ln[i]} for i in range(cnt.value)}

    def launch_count(self) -> int:
        return int(refine_ctx_launch_count(self.handle))  # noqa: F821

    def selftest_wait(self, nbytes=1024, missing=0, cycles=2_000_000, stream=None) -> int:
        """Runs the bounded-wait self-test (refine_selftest_wait) and returns
        its status code (REFINE_OK, or REFINE_ETIMEOUT when ``missing`` bytes
        never arrive)."""
        return int(refine_selftest_wait(self.handle, nbytes, missing, cycles,  # noqa: F821
                                        _stream_handle(stream, self.device)))

    def fma_rate(self, iters=1 << 17, stream=None):
        """Measured FP32 FMA throughput of the device (refine_fma_rate):
        returns (FLOP/s, ms of the timed launch)."""
        rate, ms = C.c_double(), C.c_double()
        _check(self.handle, refine_fma_rate(self.handle, int(iters), C.byref(rate), C.byref(ms),  # noqa: F821
                                            _stream_handle(stream, self.device)))
        return rate.value, ms.value

    def autotune(self, jobs, params=None, reps=3):
        """Times the batched score launch of ``jobs`` (device-tensor dicts as
        for Batch) under every candidate shape and keeps the fastest for this
        context.  Returns (best, table) as dicts."""
        arr, outs, keep = _make_jobs(self, jobs, compact=False)  # outs must outlive the call
        best = refine_shape()
        table = (refine_shape * 64)()
        cnt = C.c_int32()
        _check(self.handle, refine_autotune(self.handle, arr, len(jobs),  # noqa: F821
                                            C.byref(params) if params is not None else None, int(reps),
                                            C.byref(best), table, 64, C.byref(cnt)))
        del outs, keep
        return _shape_dict(best), [_shape_dict(table[k]) for k in range(min(cnt.value, 64))]

    def get_shape(self) -> dict:
        sh = refine_shape()
        _check(self.handle, refine_ctx_get_shape(self.handle, C.byref(sh)))  # noqa: F821
        return _shape_dict(sh)

    def set_shape(self, tile=64, cta_threads=256, ctas_per_sm=0, camera_block=512):
        sh = refine_shape(tile, cta_threads, ctas_per_sm, camera_block, 0.0)
        _check(self.handle, refine_ctx_set_shape(self.handle, C.byref(sh)))  # noqa: F821


def _make_jobs(ctx, jobs, compact=True):
    """refine_job array for device-tensor job dicts (pos, attr, cams, ratio,
    optional compact=False), with the score, mask and compaction outputs."""
    import torch
    keep, outputs = [], []
    arr = (refine_job * len(jobs))()
    for k, jd in enumerate(jobs):
        pos, attr, cams = jd["pos"], jd["attr"], jd["cams"]
        n = pos.shape[1]
        ratio = float(jd["ratio"])
        n_keep = n - int(np.floor(ratio * n))
        out = {"scores": torch.empty(n, dtype=torch.float32, device=ctx.device),
               "mask": torch.empty((n + 31) // 32, dtype=torch.int32, device=ctx.device)}
        j = arr[k]
        j.scene = make_scene(pos, attr)
        j.cams_dev = cams.data_ptr()
        j.n_views = cams.numel() // 80
        j.ratio = ratio
        j.scores_dev = out["scores"].data_ptr()
        j.keep_mask_dev = out["mask"].data_ptr()
        if compact and jd.get("compact", True):
            out["out_pos"] = torch.empty((3, max(n_keep, 1)), dtype=torch.float32, device=ctx.device)
            out["out_attr"] = empty_attr_like(attr, max(n_keep, 1), device=ctx.device)
            out["idx"] = torch.empty(max(n_keep, 1), dtype=torch.int32, device=ctx.device)
            j.out_pos_dev = out["out_pos"].data_ptr()
            j.out_attr_dev = out["out_attr"].data_ptr()
            j.out_row_stride = max(n_keep, 1)
            j.kept_idx_dev = out["idx"].data_ptr()
        out["n_keep"] = n_keep
        outputs.append(out)
        keep.append((pos, attr, cams))
    return arr, outputs, keep


def _shape_dict(sh) -> dict:
    return {"tile": sh.tile, "cta_threads": sh.cta_threads, "ctas_per_sm": sh.ctas_per_sm,
            "camera_block": sh.camera_block, "ms": sh.ms}


class Batch:
    """A batch of scenes scored by one persistent launch and replayed as a
    CUDA graph (refine_batch_*).  ``jobs`` is a list of dicts with device
    tensors: pos, attr, cams, ratio and optionally ``compact=False``.  The
    batch allocates scores, masks and compaction outputs and keeps every
    tensor alive for its lifetime."""

    def __init__(self, ctx: Context, jobs, params=None, compact=True):
        self.ctx = ctx
        arr, self.outputs, self.keep = _make_jobs(ctx, jobs, compact)
        self.n = len(jobs)
        h = C.c_void_p()
        rc = refine_batch_create(ctx.handle, arr, len(jobs), C.byref(params) if params is not None else None,  # noqa: F821
                                 C.byref(h))
        _check(ctx.handle, rc)
        self.handle = h

    def run(self, stream=None):
        _check(self.ctx.handle, refine_batch_run(self.handle, _stream_handle(stream, self.ctx.device)))  # noqa: F821

    def results(self, stream=None):
        nk = (C.c_int64 * self.n)()
        thr = (C.c_float * self.n)()
        _check(self.ctx.handle, refine_batch_results(self.handle, nk, thr,  # noqa: F821
                                                     _stream_handle(stream, self.ctx.device)))
        return list(nk), list(thr)

    def launches(self) -> int:
        return int(refine_batch_launches(self.handle))  # noqa: F821

    def close(self):
        if self.handle:
            refine_batch_destroy(self.handle)  # noqa: F821
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, MixedRows):
        if a.buf.is_cuda or a.row_stride != max(a.n, 1):
            raise ValueError("host MixedRows must be CPU rows with row stride n")
        return a.data_ptr()
    if a.is_cuda or not a.is_contiguous():
        raise ValueError("host tensors must be contiguous CPU tensors")
    return a.data_ptr()


def _host_dtype_code(a) -> int:
    if isinstance(a, MixedRows):
        return REFINE_BF16S
    if isinstance(a, np.ndarray):
        if a.dtype == np.float32:
            return REFINE_F32
        if a.dtype in (np.uint16, np.int16):
            return REFINE_BF16
    else:
        import torch
        if a.dtype == torch.float32:
            return REFINE_F32
        if a.dtype in (torch.bfloat16, torch.int16, torch.uint16):
            return REFINE_BF16
    raise TypeError(f"unsupported attribute dtype {a.dtype}")


class Queue:
    """Request queue (refine_queue_*): pruning requests for host-resident
    scenes, admitted by HBM footprint and scored in rounds by the batched
    kernel while earlier rounds run.  ``submit`` takes host arrays (numpy or
    CPU tensors; page-locked tensors are copied asynchronously) and returns a
    ticket; the queue keeps the arrays alive until ``poll`` returns them."""

    def __init__(self, ctx: Context, budget_bytes: int, max_slots: int = 8, params=None):
        self.ctx = ctx
        h = C.c_void_p()
        rc = refine_queue_create(ctx.handle, int(budget_bytes), int(max_slots),  # noqa: F821
                                 C.byref(params) if params is not None else None, C.byref(h))
        _check(ctx.handle, rc)
        self.handle = h
        self._live = {}

    @staticmethod
    def footprint(n, dtype, n_views, ratio, compact=True) -> int:
        return int(refine_queue_footprint(int(n), int(dtype), int(n_views), float(ratio), int(bool(compact))))  # noqa: F821

    def submit(self, pos, attr, cams, ratio, params=None, outputs=None, mask=True, scores=False,
               compact=True, pin=False) -> int:
        """Submits one request.  ``outputs`` may hold preallocated host
        buffers (keys mask, scores, out_pos, out_attr, idx); missing ones are
        allocated (page-locked when ``pin``)."""
        import torch
        n = int(pos.shape[1])
        dt = _host_dtype_code(attr)
        cams = np.ascontiguousarray(cams, dtype=CAMERA_DTYPE)
        n_keep = n - int(np.floor(float(ratio) * n))
        out = dict(outputs or {})

        def alloc(key, shape, np_dtype, t_dtype):
            if key not in out:
                out[key] = (torch.empty(shape, dtype=t_dtype, pin_memory=True) if pin
                            else np.empty(shape, dtype=np_dtype))
        if mask:
            alloc("mask", ((n + 31) // 32,), np.uint32, torch.int32)
        if scores:
            alloc("scores", (n,), np.float32, torch.float32)
        if compact:
            alloc("out_pos", (3, n_keep), np.float32, torch.float32)
            if dt == REFINE_BF16S:
                if "out_attr" not in out:
                    out["out_attr"] = MixedRows.empty(n_keep, pin_memory=pin)
            else:
                alloc("out_attr", (56, n_keep), np.float32 if dt == REFINE_F32 else np.uint16,
                      torch.float32 if dt == REFINE_F32 else torch.bfloat16)
            alloc("idx", (n_keep,), np.int32, torch.int32)
        r = refine_request()
        r.n = n
        r.dtype = dt
        r.n_views = len(cams)
        r.pos_host = _host_ptr(pos)
        r.attr_host = _host_ptr(attr)
        r.cams_host = cams.ctypes.data
        r.ratio = float(ratio)
        r.params = C.cast(C.pointer(params), C.c_void_p) if params is not None else None
        r.keep_mask_host = _host_ptr(out.get("mask"))
        r.scores_host = _host_ptr(out.get("scores"))
        r.out_pos_host = _host_ptr(out.get("out_pos"))
        r.out_attr_host = _host_ptr(out.get("out_attr"))
        r.kept_idx_host = _host_ptr(out.get("idx"))
        t = C.c_uint64()
        rc = refine_queue_submit(self.handle, C.byref(r), C.byref(t))  # noqa: F821
        if rc != REFINE_OK:
            raise RefineError(rc, f"refine_queue_submit: {STATUS_NAMES.get(rc, rc)}")
        self._live[t.value] = (pos, attr, cams, out)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns (result dict, outputs dict) or None if not done in time."""
        res = refine_result()
        rc = refine_queue_poll(self.handle, int(ticket), C.byref(res), int(timeout_ms))  # noqa: F821
        if rc == REFINE_ETIMEOUT:
            return None
        if rc != REFINE_OK:
            raise RefineError(rc, f"refine_queue_poll: {STATUS_NAMES.get(rc, rc)}")
        _, _, _, out = self._live.pop(int(ticket))
        d = {k: getattr(res, k) for k, _ in refine_result._fields_ if k != "reserved"}
        return d, out

    def poll_any(self, timeout_ms: int = -1):
        """The first request to finish: (ticket, result dict, outputs dict),
        or None if none is done in time (refine_queue_poll_any)."""
        res = refine_result()
        t = C.c_uint64()
        rc = refine_queue_poll_any(self.handle, C.byref(t), C.byref(res), int(timeout_ms))  # noqa: F821
        if rc == REFINE_ETIMEOUT:
            return None
        if rc != REFINE_OK:
            raise RefineError(rc, f"refine_queue_poll_any: {STATUS_NAMES.get(rc, rc)}")
        _, _, _, out = self._live.pop(int(t.value))
        d = {k: getattr(res, k) for k, _ in refine_result._fields_ if k != "reserved"}
        return int(t.value), d, out

    def last_error(self) -> str:
        return refine_queue_last_error(self.handle).decode(errors="replace")  # noqa: F821

    def stats(self) -> dict:
        st = refine_queue_stats()
        refine_queue_stats_get(self.handle, C.byref(st))  # noqa: F821
        return {k: getattr(st, k) for k, _ in refine_queue_stats._fields_}

    def close(self):
        if self.handle:
            refine_queue_destroy(self.handle)  # noqa: F821
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def write_ply(path: str, pos, attr) -> None:
    """Writes host rows pos [3, n] float32 and attr [56, n] (float32 or
    bfloat16 bits as uint16, or host MixedRows) as a 3DGS scene PLY
    (refine_write_ply)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    if isinstance(attr, MixedRows):
        if attr.buf.is_cuda:
            raise ValueError("write_ply takes host rows")
        rc = refine_write_ply(os.fsencode(path), attr.n, REFINE_BF16S, pos.ctypes.data,  # noqa: F821
                              attr.data_ptr(), attr.row_stride)
        if rc != REFINE_OK:
            raise RefineError(rc, f"refine_write_ply: cannot write {path}")
        return
    attr = np.ascontiguousarray(attr)
    dt = REFINE_F32 if attr.dtype == np.float32 else REFINE_BF16
    if dt == REFINE_BF16 and attr.dtype not in (np.uint16, np.int16):
        raise TypeError("attr must be float32 or bfloat16 bits (uint16)")
    n = pos.shape[1]
    rc = refine_write_ply(os.fsencode(path), n, dt, pos.ctypes.data, attr.ctypes.data, n)  # noqa: F821
    if rc != REFINE_OK:
        raise RefineError(rc, f"refine_write_ply: cannot write {path}")


def read_ply(path: str):
    """Reads a 3DGS scene PLY into (pos [3, n], attr [56, n]) float32."""
    n = C.c_int64()
    rc = refine_read_ply(os.fsencode(path), C.byref(n), None, None, 0)  # noqa: F821
    if rc != REFINE_OK:
        raise RefineError(rc, f"refine_read_ply: {path} is not a scene PLY")
    pos = np.empty((3, n.value), dtype=np.float32)
    attr = np.empty((56, n.value), dtype=np.float32)
    rc = refine_read_ply(os.fsencode(path), C.byref(n), pos.ctypes.data, attr.ctypes.data, n.value)  # noqa: F821
    if rc != REFINE_OK:
        raise RefineError(rc, f"refine_read_ply: {path}")
    return pos, attr
