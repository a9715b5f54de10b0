"""Python access to the FP64 CPU oracle (``refine_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package.  It does
not import the CUDA library and the CUDA library never imports it.

The shared object is built with plain gcc (``-O2 -fopenmp``, no SIMD
intrinsics) into ``oracle/_build/liboracle.so`` on first use, or by
``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "refine_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

NO_VIS = 1 << 0
NO_PROJ = 1 << 1
EQUAL_LAMBDA = 1 << 2
NORM_ATTR = 1 << 3
FULL_JACOBIAN = 1 << 4

# Calibration constants of Eq. 18 (E[ln F_gem], E[F_col], E[F_opa]); see
# ``calibrate.py`` for how they were produced.
from .calibration import E_LN_GEM, E_COL, E_OPA  # noqa: E402

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the path of the shared object."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_double), ("height", C.c_double), ("znear", C.c_double),
                ("zfar", C.c_double)]


class Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("e_ln_gem", C.c_double), ("e_col", C.c_double),
                ("e_opa", C.c_double), ("luma", C.c_double * 3), ("flags", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("F_col", C.c_double), ("F_opa", C.c_double), ("F_gem", C.c_double),
                ("lambda_t", C.c_double * 3), ("lambda_", C.c_double * 3),
                ("mean_m", C.c_double * 3)]

    def as_dict(self):
        return {"F_col": self.F_col, "F_opa": self.F_opa, "F_gem": self.F_gem,
                "lambda_t": list(self.lambda_t), "lambda": list(self.lambda_),
                "mean_m": list(self.mean_m)}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            i64 = C.c_int64
            L.orc_activate.argtypes = [dp, i64, i64, dp, dp, dp, dp]
            L.orc_to_camera.argtypes = [C.POINTER(Camera), dp, dp]
            L.orc_project.argtypes = [C.POINTER(Camera), dp, dp]
            L.orc_projection_jacobian.argtypes = [C.POINTER(Camera), dp, dp]
            L.orc_cov2d.argtypes = [C.POINTER(Camera), dp, dp, dp]
            L.orc_visible.argtypes = [C.POINTER(Camera), dp, dp, C.POINTER(C.c_int)]
            L.orc_visible.restype = C.c_int
            L.orc_magnitudes.argtypes = [dp, i64, i64, dp]
            L.orc_scene_stats.argtypes = [dp, i64, i64, C.POINTER(Params), C.POINTER(Stats)]
            L.orc_score.argtypes = [dp, i64, i64, C.POINTER(Camera), C.c_int, C.POINTER(Params),
                                    dp, dp, dp, C.POINTER(C.c_int32), dp, C.POINTER(Stats)]
            L.orc_score_subset.argtypes = [dp, i64, i64, C.POINTER(C.c_int64), i64,
                                           C.POINTER(Camera), C.c_int, C.POINTER(Params),
                                           dp, dp, dp, C.POINTER(C.c_int32), dp, C.POINTER(Stats)]
            L.orc_select.argtypes = [dp, i64, C.c_double, C.POINTER(C.c_uint32), dp]
            L.orc_select.restype = i64
            L.orc_compact.argtypes = [C.c_void_p, i64, i64, C.c_int, C.c_int,
                                      C.POINTER(C.c_uint32), C.c_void_p, i64,
                                      C.POINTER(C.c_int32)]
            L.orc_compact.restype = i64
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def cameras(cams) -> "C.Array":
    """Convert a ``synth.CAMERA_DTYPE`` array (float32 fields) to oracle
    cameras; every value is widened exactly to double."""
    arr = (Camera * max(len(cams), 1))()
    for k, c in enumerate(cams):
        o = arr[k]
        o.R[:] = [float(x) for x in np.asarray(c["R"], dtype=np.float64)]
        o.t[:] = [float(x) for x in np.asarray(c["t"], dtype=np.float64)]
        o.fx, o.fy, o.cx, o.cy = (float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"]))
        o.width, o.height = float(c["width"]), float(c["height"])
        o.znear, o.zfar = float(c["znear"]), float(c["zfar"])
    return arr


def params(eta=0.05, e_ln_gem=None, e_col=None, e_opa=None,
           luma=(0.299, 0.587, 0.114), flags=NORM_ATTR) -> Params:
    p = Params()
    p.eta = eta
    p.e_ln_gem = E_LN_GEM if e_ln_gem is None else e_ln_gem
    p.e_col = E_COL if e_col is None else e_col
    p.e_opa = E_OPA if e_opa is None else e_opa
    p.luma[:] = list(luma)
    p.flags = flags
    return p


def set_threads(k: int) -> None:
    lib().orc_set_num_threads(int(k))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ------------------------------------------------------- per-item helpers

def activate(g: np.ndarray, i: int):
    g = np.ascontiguousarray(g, dtype=np.float64)
    a = C.c_double()
    s = np.zeros(3); R = np.zeros(9); S = np.zeros(9)
    lib().orc_activate(_dp(g), g.shape[1], i, C.byref(a), _dp(s), _dp(R), _dp(S))
    return a.value, s, R.reshape(3, 3), S.reshape(3, 3)


def magnitudes(g: np.ndarray, i: int) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float64)
    m = np.zeros(3)
    lib().orc_magnitudes(_dp(g), g.shape[1], i, _dp(m))
    return m


def to_camera(cam: Camera, mu) -> np.ndarray:
    mu = np.ascontiguousarray(mu, dtype=np.float64); out = np.zeros(3)
    lib().orc_to_camera(C.byref(cam), _dp(mu), _dp(out))
    return out


def project(cam: Camera, tc) -> np.ndarray:
    tc = np.ascontiguousarray(tc, dtype=np.float64); out = np.zeros(2)
    lib().orc_project(C.byref(cam), _dp(tc), _dp(out))
    return out


def jacobian(cam: Camera, tc) -> np.ndarray:
    tc = np.ascontiguousarray(tc, dtype=np.float64); out = np.zeros(6)
    lib().orc_projection_jacobian(C.byref(cam), _dp(tc), _dp(out))
    return out.reshape(2, 3)


def cov2d(cam: Camera, tc, Sigma) -> np.ndarray:
    tc = np.ascontiguousarray(tc, dtype=np.float64)
    S = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(9)
    out = np.zeros(4)
    lib().orc_cov2d(C.byref(cam), _dp(tc), _dp(S), _dp(out))
    return out.reshape(2, 2)


def visible(cam: Camera, mu, Sigma):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    S = np.ascontiguousarray(Sigma, dtype=np.float64).reshape(9)
    b = C.c_int()
    v = lib().orc_visible(C.byref(cam), _dp(mu), _dp(S), C.byref(b))
    return bool(v), bool(b.value)


# ---------------------------------------------------------- whole passes

def scene_stats(g: np.ndarray, p: Params | None = None) -> dict:
    g = np.ascontiguousarray(g, dtype=np.float64)
    st = Stats()
    lib().orc_scene_stats(_dp(g), g.shape[1], g.shape[1], C.byref(p or params()), C.byref(st))
    return st.as_dict()


def score(g: np.ndarray, cams, p: Params | None = None, detail: bool = True) -> dict:
    """Scores of every primitive of the FP64 parameter block ``g`` [59, n].

    Returns ``scores``, and with ``detail``: ``S`` (visibility-weighted view
    sum), ``S_sure`` (the sum over pairs outside the parity band),
    ``nborder`` and ``bterms`` (up to four borderline terms per primitive)
    and the scene ``stats``."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    n = g.shape[1]
    camarr = cams if isinstance(cams, C.Array) else cameras(cams)
    V = len(cams)
    out = {"scores": np.zeros(n)}
    S = np.zeros(n) if detail else None
    Ss = np.zeros(n) if detail else None
    nb = np.zeros(n, dtype=np.int32) if detail else None
    bt = np.zeros((n, 4)) if detail else None
    st = Stats()
    lib().orc_score(_dp(g), n, n, camarr, V, C.byref(p or params()), _dp(out["scores"]),
                    _dp(S) if detail else None, _dp(Ss) if detail else None,
                    nb.ctypes.data_as(C.POINTER(C.c_int32)) if detail else None,
                    _dp(bt) if detail else None, C.byref(st))
    out["stats"] = st.as_dict()
    if detail:
        out.update(S=S, S_sure=Ss, nborder=nb, bterms=bt)
    return out


def score_subset(g: np.ndarray, idx: np.ndarray, cams, p: Params | None = None) -> dict:
    """Like ``score`` for the primitives ``idx`` only; the scene statistics
    (lambda, magnitude means) still come from every column of ``g``."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.shape[0]
    camarr = cams if isinstance(cams, C.Array) else cameras(cams)
    o = {"scores": np.zeros(m), "S": np.zeros(m), "S_sure": np.zeros(m),
         "nborder": np.zeros(m, dtype=np.int32), "bterms": np.zeros((m, 4))}
    st = Stats()
    lib().orc_score_subset(_dp(g), g.shape[1], g.shape[1], idx.ctypes.data_as(C.POINTER(C.c_int64)),
                           m, camarr, len(cams), C.byref(p or params()), _dp(o["scores"]),
                           _dp(o["S"]), _dp(o["S_sure"]),
                           o["nborder"].ctypes.data_as(C.POINTER(C.c_int32)), _dp(o["bterms"]),
                           C.byref(st))
    o["stats"] = st.as_dict()
    return o


def select(scores: np.ndarray, beta: float):
    """Ratio pruning of Sec. 3.3.  Returns (mask words uint32, threshold, n_keep)."""
    s = np.ascontiguousarray(scores, dtype=np.float64)
    n = s.shape[0]
    mask = np.zeros(max((n + 31) // 32, 1), dtype=np.uint32)
    thr = C.c_double()
    nk = lib().orc_select(_dp(s), n, float(beta), mask.ctypes.data_as(C.POINTER(C.c_uint32)),
                          C.byref(thr))
    return mask[: (n + 31) // 32], thr.value, int(nk)


def compact(rows: np.ndarray, mask: np.ndarray, out_stride: int | None = None):
    """Stable gather of kept columns of ``rows`` [r, n] (any element size).
    Returns (kept rows [r, n_keep], kept indices int32)."""
    rows = np.ascontiguousarray(rows)
    r, n = rows.shape
    nk = int(sum(bin(int(w)).count("1") for w in mask)) if n else 0
    stride = out_stride or max(nk, 1)
    out = np.zeros((r, stride), dtype=rows.dtype)
    idx = np.zeros(max(nk, 1), dtype=np.int32)
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    if m.size == 0:
        m = np.zeros(1, dtype=np.uint32)
    got = lib().orc_compact(rows.ctypes.data, n, n, r, rows.dtype.itemsize,
                            m.ctypes.data_as(C.POINTER(C.c_uint32)), out.ctypes.data,
                            stride, idx.ctypes.data_as(C.POINTER(C.c_int32)))
    return out[:, :got], idx[:got]


def valid_alternative(S_gpu: np.ndarray, o: dict, rtol: float) -> np.ndarray:
    """For primitives with borderline pairs: does the GPU view sum equal
    S_sure plus some subset of the borderline terms (each borderline pair may
    be decided either way), within ``rtol``?  Primitives with more than four
    borderline pairs are accepted when S_gpu lies between S_sure and
    S_sure + all terms.  Returns a boolean array over all primitives (True
    where there is nothing to check)."""
    ok = np.ones(S_gpu.shape[0], dtype=bool)
    for i in np.nonzero(o["nborder"])[0]:
        k = int(o["nborder"][i])
        base = o["S_sure"][i]
        terms = o["bterms"][i, : min(k, 4)]
        s = float(S_gpu[i])
        if k > 4:
            ok[i] = base * (1 - rtol) <= s
            continue
        found = False
        for mask in range(1 << len(terms)):
            cand = base + sum(terms[b] for b in range(len(terms)) if mask >> b & 1)
            if abs(s - cand) <= rtol * max(abs(cand), 1e-30):
                found = True
                break
        ok[i] = found
    return ok

