"""Thin Python binding of include/dco_stereo.h (ctypes, argument marshalling only).

Every step of the matcher runs in libdco_stereo.so; this module converts
torch tensors / numpy arrays to pointers and sizes, nothing else.  Method
names mirror the C entry points: dco_stereo_<name> -> Stereo.<name>.

There is no fallback: if the library is not built, or no CUDA device is
present, constructing a Stereo raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import NamedTuple, Optional, Sequence

import numpy as np

from . import build as _build

c_int, c_float, c_void_p, c_size_t = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t

STATUS = {0: "DCO_OK", 1: "DCO_EINVAL", 2: "DCO_ENOMEM", 3: "DCO_EBUDGET", 4: "DCO_ECUDA",
          5: "DCO_ETIMEOUT", 6: "DCO_EDEVICE"}
DCO_OK, DCO_EINVAL, DCO_ENOMEM, DCO_EBUDGET, DCO_ECUDA, DCO_ETIMEOUT, DCO_EDEVICE = range(7)
DCO_TEST_LOSE_TILE_COPIES = 1   # failure test flags (include/dco_stereo.h)
DCO_TEST_LOSE_GRID_ARRIVAL = 4


class Params(ctypes.Structure):
    """dco_params; defaults from dco_params_default()."""
    _fields_ = [("lambda_ad", c_float), ("lambda_census", c_float), ("gamma_l", c_float),
                ("eps", c_float), ("census_w", c_int), ("census_h", c_int), ("arm_l1", c_int),
                ("arm_l2", c_int), ("tau1", c_int), ("tau2", c_int), ("lr_tol", c_int),
                ("d_chunk", c_int), ("vote_iters", c_int), ("smooth_arms", c_int),
                ("agg_order", c_int), ("d_min", c_int), ("h_chunk", c_int), ("v_chunk", c_int)]

    @classmethod
    def default(cls, **over) -> "Params":
        p = cls()
        _check(lib().dco_params_default(ctypes.byref(p)), None)
        for k, v in over.items():
            setattr(p, k, v)
        return p


class DenseParams(ctypes.Structure):
    """dco_dense_params; defaults from dco_dense_params_default()."""
    _fields_ = [("lambda_d", c_float), ("lambda_s", c_float), ("lambda_s2", c_float), ("tol", c_float),
                ("max_iters", c_int), ("solver", c_int)]

    @classmethod
    def default(cls, **over) -> "DenseParams":
        p = cls()
        _check(lib().dco_dense_params_default(ctypes.byref(p)), None)
        for k, v in over.items():
            setattr(p, k, v)
        return p


class Tile(NamedTuple):
    """Per-shape tile choice: the pass width (disparities per pass) and the
    blocks of the two 1-D passes (dco_params.d_chunk, h_chunk, v_chunk);
    0 = the call's parameters."""
    d_chunk: int = 0
    h_chunk: int = 0
    v_chunk: int = 0

    @classmethod
    def of(cls, v) -> "Tile":
        """A Tile from None, a pass width alone or a (d, h, v) sequence."""
        if v is None:
            return cls()
        if isinstance(v, (int, np.integer)):
            return cls(int(v))
        return cls(*(int(x) for x in v))

    def apply(self, p: "Params") -> "Params":
        """p with this tile's nonzero fields set."""
        for k, v in zip(self._fields, self):
            if v:
                setattr(p, k, v)
        return p


class PairDesc(ctypes.Structure):
    _fields_ = [("left", c_void_p), ("right", c_void_p), ("W", c_int), ("H", c_int), ("D", c_int),
                ("disp_out", c_void_p), ("d_chunk", c_int), ("h_chunk", c_int), ("v_chunk", c_int)]


class StreamDesc(ctypes.Structure):
    _fields_ = [("W", c_int), ("H", c_int), ("D", c_int), ("d_chunk", c_int), ("h_chunk", c_int),
                ("v_chunk", c_int), ("priority", c_int)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("launch_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("device_ms", c_float)]


class DcoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/dco_stereo.h declares."""
    text = open(os.path.join(_build.INCLUDE, "dco_stereo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dco_\w+)\s*\(", text)))


def lib():
    """The loaded libdco_stereo.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P = c_void_p
        sig = {
            "dco_params_default": (c_int, [P]),
            "dco_status_string": (ctypes.c_char_p, [c_int]),
            "dco_stereo_create": (c_int, [P, c_int, c_size_t]),
            "dco_stereo_destroy": (None, [P]),
            "dco_stereo_workspace_bytes": (c_size_t, [c_int, c_int, c_int, P]),
            "dco_stereo_reserve": (c_int, [P, c_int, c_int, c_int, P]),
            "dco_stereo_match": (c_int, [P, P, P, c_int, c_int, c_int, P, P, P]),
            "dco_stereo_match_views": (c_int, [P, P, P, c_int, c_int, c_int, P, P, P, P, P, P, P]),
            "dco_stereo_match_host": (c_int, [P, P, P, c_int, c_int, c_int, P, P, P]),
            "dco_stereo_census": (c_int, [P, P, c_int, c_int, P, P, P]),
            "dco_stereo_arms": (c_int, [P, P, c_int, c_int, P, P, P]),
            "dco_stereo_cost_volume": (c_int, [P, P, P, c_int, c_int, c_int, P, c_int, P, P]),
            "dco_stereo_lr_check": (c_int, [P, P, P, c_int, c_int, c_int, P, P]),
            "dco_stereo_vote": (c_int, [P, P, P, c_int, c_int, c_int, P, P, P]),
            "dco_stereo_downscale": (c_int, [P, P, c_int, c_int, P, P]),
            "dco_dense_params_default": (c_int, [P]),
            "dco_stereo_densify": (c_int, [P, P, P, P, P, P, c_int, c_int, P, P, P]),
            "dco_stereo_densify_stats": (c_int, [P, P, P]),
            "dco_stereo_depth": (c_int, [P, P, P, c_int, c_int, c_int, P, ctypes.c_double, ctypes.c_double, P, P,
                                         P]),
            "dco_stereo_match_batch": (c_int, [P, P, c_int, P, P]),
            "dco_stereo_sync_status": (c_int, [P]),
            "dco_stereo_last_error": (ctypes.c_char_p, [P]),
            "dco_stereo_set_profiling": (c_int, [P, c_int]),
            "dco_stereo_profile_reset": (c_int, [P]),
            "dco_stereo_profile_count": (c_int, [P]),
            "dco_stereo_profile_get": (c_int, [P, c_int, P, P, P]),
            "dco_stereo_launch_count": (ctypes.c_ulonglong, [P]),
            "dco_stereo_match_noalloc": (c_int, [P, P, c_int, c_int, c_int, P, P, P]),
            "dco_stereo_noalloc_status": (c_int, [P]),
            "dco_stereo_stream_status": (c_int, [P, P]),
            "dco_stereo_set_test_flags": (c_int, [P, c_int]),
            "dco_stereo_workspace_allocated": (c_size_t, [P]),
            "dco_stereo_batch_groups": (c_int, [P]),
            "dco_server_create": (c_int, [P, c_int, P, c_int, c_int, c_int, c_int, c_size_t, P]),
            "dco_server_submit": (c_int, [P, c_int, P, P, P, P]),
            "dco_server_wait": (c_int, [P, ctypes.c_ulonglong, c_int, P]),
            "dco_server_counters": (c_int, [P, P, P, P, P]),
            "dco_server_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, h) -> None:
    if code != DCO_OK:
        detail = ""
        if h is not None:
            detail = (lib().dco_stereo_last_error(h) or b"").decode()
        raise DcoError(code, (lib().dco_status_string(code) or b"").decode() + (f" ({detail})" if detail else ""))


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    """The cudaStream_t of `stream` (None: torch's current stream on the
    current device)."""
    if stream is None:
        import torch
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(torch._C, "_cuda_getDevice", None)
        if raw is not None and dev is not None:   # the same stream, without a Stream object (0.2 against 3 us)
            return raw(dev())
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _is_np(t) -> bool:
    return isinstance(t, np.ndarray)


def _contiguous(t) -> bool:
    return t.flags.c_contiguous if _is_np(t) else t.is_contiguous()


_NP_DTYPES = {n: np.dtype(n) for n in ("uint8", "int16", "float32", "int64")}


def _dtype_ok(t, name: str) -> bool:
    """t's element type is `name` ("uint8", "int16", "float32", "int64")."""
    if _is_np(t):
        return t.dtype == _NP_DTYPES[name]
    import torch
    return t.dtype == getattr(torch, name)


def _expect(what: str, t, shape, dtype: str, like=None) -> None:
    """Raise ValueError unless `t` is a contiguous (H, W, ...) buffer of the
    given shape and element type, on the same device as `like` (a torch
    tensor) when given.  The library trusts the sizes it is passed, so a
    buffer of the wrong size would be read or written out of bounds."""
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not _dtype_ok(t, dtype):
        raise ValueError(f"{what}: element type {t.dtype}, expected {dtype}")
    if not _contiguous(t):
        raise ValueError(f"{what}: must be contiguous")
    if like is not None and not _is_np(t) and t.device != like.device:
        raise ValueError(f"{what}: on {t.device}, expected {like.device}")


def _rgb_dims(t) -> tuple[int, int]:
    """(W, H) of an (H, W, 3) uint8 contiguous image (array or tensor)."""
    if len(t.shape) != 3 or int(t.shape[2]) != 3:
        raise ValueError(f"images are (H, W, 3) uint8, got shape {tuple(t.shape)}")
    _expect("image", t, t.shape, "uint8")
    return int(t.shape[1]), int(t.shape[0])


class Stereo:
    """A dco_stereo handle on one CUDA device (owns the workspace)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self._h = c_void_p()
        _check(lib().dco_stereo_create(ctypes.byref(self._h), device, budget_bytes), None)
        self.device = device

    def close(self) -> None:
        if self._h:
            lib().dco_stereo_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- sizing
    @staticmethod
    def workspace_bytes(W: int, H: int, D: int, params: Optional[Params] = None) -> int:
        return int(lib().dco_stereo_workspace_bytes(W, H, D, ctypes.byref(params) if params else None))

    def reserve(self, W: int, H: int, D: int, params: Optional[Params] = None) -> None:
        _check(lib().dco_stereo_reserve(self._h, W, H, D, ctypes.byref(params) if params else None), self._h)

    # -- the hot path
    def match(self, left, right, D: int, params: Optional[Params] = None, out=None, stream=None):
        import torch
        W, H = _rgb_dims(left)
        _expect("right", right, left.shape, "uint8", left)
        if out is None:
            out = torch.empty((H, W), dtype=torch.int16, device=left.device)
        _expect("out", out, (H, W), "int16", left)
        _check(lib().dco_stereo_match(self._h, _ptr(left), _ptr(right), W, H, D,
                                      ctypes.byref(params) if params else None, _ptr(out),
                                      _stream(stream)), self._h)
        return out

    def match_views(self, left, right, D: int, params: Optional[Params] = None, stream=None,
                    costs: bool = True):
        import torch
        W, H = _rgb_dims(left)
        _expect("right", right, left.shape, "uint8", left)
        dev = left.device
        out = torch.empty((H, W), dtype=torch.int16, device=dev)
        dl = torch.empty_like(out)
        dr = torch.empty_like(out)
        cl = torch.empty((H, W), dtype=torch.float32, device=dev) if costs else None
        cr = torch.empty((H, W), dtype=torch.float32, device=dev) if costs else None
        _check(lib().dco_stereo_match_views(self._h, _ptr(left), _ptr(right), W, H, D,
                                            ctypes.byref(params) if params else None, _ptr(out),
                                            _ptr(dl), _ptr(dr), _ptr(cl), _ptr(cr), _stream(stream)),
               self._h)
        return out, dl, dr, cl, cr

    def match_host(self, left: np.ndarray, right: np.ndarray, D: int,
                   params: Optional[Params] = None, out: Optional[np.ndarray] = None, stream=None):
        W, H = _rgb_dims(left)
        _expect("right", right, left.shape, "uint8")
        if out is None:
            out = np.empty((H, W), np.int16)
        _expect("out", out, (H, W), "int16")
        _check(lib().dco_stereo_match_host(self._h, _ptr(left), _ptr(right), W, H, D,
                                           ctypes.byref(params) if params else None, _ptr(out),
                                           _stream(stream)), self._h)
        return out

    def match_batch(self, pairs: Sequence, params: Optional[Params] = None, stream=None):
        """pairs: sequence of (left, right, D, out) device tensors, or
        (left, right, D, out, tile) with the pair's own pass width (an int)
        or Tile (pass width and blocks)."""
        arr = (PairDesc * len(pairs))()
        for i, pr in enumerate(pairs):
            l, r, D, o = pr[:4]
            t = Tile.of(pr[4] if len(pr) > 4 else None)
            W, H = _rgb_dims(l)
            _expect(f"pair {i} right", r, l.shape, "uint8", l)
            _expect(f"pair {i} out", o, (H, W), "int16", l)
            arr[i] = PairDesc(_ptr(l), _ptr(r), W, H, D, _ptr(o), *t)
        _check(lib().dco_stereo_match_batch(self._h, arr, len(pairs),
                                            ctypes.byref(params) if params else None, _stream(stream)),
               self._h)

    # -- stages
    def census(self, img, params: Optional[Params] = None, stream=None):
        import torch
        W, H = _rgb_dims(img)
        out = torch.empty((H, W), dtype=torch.int64, device=img.device)
        _check(lib().dco_stereo_census(self._h, _ptr(img), W, H, ctypes.byref(params) if params else None,
                                       _ptr(out), _stream(stream)), self._h)
        return out

    def arms(self, img, params: Optional[Params] = None, stream=None):
        import torch
        W, H = _rgb_dims(img)
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=img.device)
        _check(lib().dco_stereo_arms(self._h, _ptr(img), W, H, ctypes.byref(params) if params else None,
                                     _ptr(out), _stream(stream)), self._h)
        return out

    def cost_volume(self, left, right, D: int, view: int, params: Optional[Params] = None, stream=None):
        import torch
        W, H = _rgb_dims(left)
        _expect("right", right, left.shape, "uint8", left)
        out = torch.empty((D, H, W), dtype=torch.float32, device=left.device)
        _check(lib().dco_stereo_cost_volume(self._h, _ptr(left), _ptr(right), W, H, D,
                                            ctypes.byref(params) if params else None, view, _ptr(out),
                                            _stream(stream)), self._h)
        return out

    def lr_check(self, dl, dr, tol: int = 1, stream=None):
        import torch
        if len(dl.shape) != 2:
            raise ValueError(f"dl: an (H, W) int16 map, got shape {tuple(dl.shape)}")
        H, W = dl.shape
        _expect("dl", dl, (H, W), "int16")
        _expect("dr", dr, (H, W), "int16", dl)
        out = torch.empty_like(dl)
        _check(lib().dco_stereo_lr_check(self._h, _ptr(dl), _ptr(dr), W, H, tol, _ptr(out),
                                         _stream(stream)), self._h)
        return out

    def vote(self, img, disp, D: int, params: Optional[Params] = None, out=None, stream=None):
        """params.vote_iters rounds of the Eq. 4 parallax optimisation of the
        int16 map `disp` over the support regions of `img` (device tensors)."""
        import torch
        W, H = _rgb_dims(img)
        _expect("disp", disp, (H, W), "int16", img)
        if out is None:
            out = torch.empty_like(disp)
        _expect("out", out, (H, W), "int16", img)
        _check(lib().dco_stereo_vote(self._h, _ptr(img), _ptr(disp), W, H, D,
                                     ctypes.byref(params) if params else None, _ptr(out), _stream(stream)),
               self._h)
        return out

    def densify(self, d_sparse, contour=None, m_fuse=None, m_int=None, d_pre=None,
                params: Optional[DenseParams] = None, out=None, stream=None):
        """Dense depth (Sect. 6, Eq. 20) from device float maps (H, W); returns
        the output tensor (the call waits for the solve)."""
        import torch
        if len(d_sparse.shape) != 2:
            raise ValueError(f"d_sparse: an (H, W) float32 map, got shape {tuple(d_sparse.shape)}")
        H, W = d_sparse.shape
        _expect("d_sparse", d_sparse, (H, W), "float32")
        for what, t, dt in (("contour", contour, "uint8"), ("m_fuse", m_fuse, "float32"),
                            ("m_int", m_int, "float32"), ("d_pre", d_pre, "float32")):
            if t is not None:
                _expect(what, t, (H, W), dt, d_sparse)
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=d_sparse.device)
        _expect("out", out, (H, W), "float32", d_sparse)
        opt = lambda t: _ptr(t) if t is not None else None
        _check(lib().dco_stereo_densify(self._h, _ptr(d_sparse), opt(contour), opt(m_fuse), opt(m_int),
                                        opt(d_pre), W, H, ctypes.byref(params) if params else None, _ptr(out),
                                        _stream(stream)), self._h)
        return out

    def densify_stats(self) -> tuple[int, float]:
        it, rr = c_int(0), ctypes.c_double(0.0)
        _check(lib().dco_stereo_densify_stats(self._h, ctypes.byref(it), ctypes.byref(rr)), self._h)
        return it.value, rr.value

    def downscale(self, img, stream=None):
        import torch
        W, H = _rgb_dims(img)
        out = torch.empty((H // 2, W // 2, 3), dtype=torch.uint8, device=img.device)
        _check(lib().dco_stereo_downscale(self._h, _ptr(img), W, H, _ptr(out), _stream(stream)), self._h)
        return out

    def depth(self, left, right, D: int, f_px: float, baseline: float, params: Optional[Params] = None,
              out=None, disp_half=None, stream=None):
        """Full-size sparse depth (float32, 0 = missing) from a full-size pair
        matched at half of each axis over D disparities."""
        import torch
        W, H = _rgb_dims(left)
        _expect("right", right, left.shape, "uint8", left)
        if out is None:
            out = torch.empty((H, W), dtype=torch.float32, device=left.device)
        _expect("out", out, (H, W), "float32", left)
        if disp_half is not None:
            _expect("disp_half", disp_half, (H // 2, W // 2), "int16", left)
        _check(lib().dco_stereo_depth(self._h, _ptr(left), _ptr(right), W, H, D,
                                      ctypes.byref(params) if params else None, float(f_px), float(baseline),
                                      _ptr(out), _ptr(disp_half) if disp_half is not None else None,
                                      _stream(stream)), self._h)
        return out

    # -- status and profiling
    def sync_status(self) -> None:
        _check(lib().dco_stereo_sync_status(self._h), self._h)

    def stream_status(self, stream=None) -> None:
        """Status word read in order on `stream` (waits for that stream only)."""
        _check(lib().dco_stereo_stream_status(self._h, _stream(stream)), self._h)

    def set_test_flags(self, flags: int) -> None:
        _check(lib().dco_stereo_set_test_flags(self._h, int(flags)), self._h)

    def workspace_allocated(self) -> int:
        return int(lib().dco_stereo_workspace_allocated(self._h))

    def batch_groups(self) -> int:
        return int(lib().dco_stereo_batch_groups(self._h))

    def set_profiling(self, on: bool) -> None:
        _check(lib().dco_stereo_set_profiling(self._h, 1 if on else 0), self._h)

    def profile_reset(self) -> None:
        _check(lib().dco_stereo_profile_reset(self._h), self._h)

    def launch_count(self) -> int:
        return int(lib().dco_stereo_launch_count(self._h))

    def profile(self) -> dict:
        """{kernel name: (launches, total ms)} since the last reset."""
        n = lib().dco_stereo_profile_count(self._h)
        res = {}
        for i in range(n):
            name = ctypes.c_char_p()
            cnt = c_int()
            ms = ctypes.c_double()
            _check(lib().dco_stereo_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(cnt),
                                                ctypes.byref(ms)), self._h)
            res[name.value.decode()] = (cnt.value, ms.value)
        return res


class NativeServer:
    """The library's serving runtime (dco_server_*): continuous batching of
    frames from several camera streams, scheduled and retired by native
    threads.  submit() takes host uint8 (H, W, 3) images and an int16 (H, W)
    output buffer of the stream's shape (pinned numpy arrays make the copies
    asynchronous) and returns a ticket; wait(ticket) blocks until the map is
    in the output buffer and returns the request's times."""

    def __init__(self, shapes, device: int = 0, lanes: int = 2, slots_per_stream: int = 3, max_batch: int = 16,
                 budget_bytes: int = 0, params: Optional[Params] = None, tiles=None, priorities=None):
        """priorities: per stream 1 = latency-critical (admitted first, run on
        high-priority CUDA streams), 0 = normal; "smaller" marks every
        stream whose frames are smaller (W x H x D) than the largest."""
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        ts = [Tile.of(v) for v in (tiles or [None] * len(self.shapes))]
        if priorities == "smaller":
            big = max(W * H * D for W, H, D in self.shapes)
            priorities = [int(W * H * D < big) for W, H, D in self.shapes]
        pr = [int(v) for v in (priorities or [0] * len(self.shapes))]
        arr = (StreamDesc * len(self.shapes))(*[StreamDesc(W, H, D, *t, q)
                                                for (W, H, D), t, q in zip(self.shapes, ts, pr)])
        self._s = c_void_p()
        self._keep = {}
        _check(lib().dco_server_create(ctypes.byref(self._s), device, arr, len(self.shapes), lanes, slots_per_stream,
                                       max_batch, budget_bytes, ctypes.byref(params) if params else None), None)

    def submit(self, stream: int, left: np.ndarray, right: np.ndarray, out: np.ndarray) -> int:
        W, H, _ = self.shapes[stream]
        _expect("left", left, (H, W, 3), "uint8")
        _expect("right", right, (H, W, 3), "uint8")
        _expect("out", out, (H, W), "int16")
        t = ctypes.c_ulonglong()
        _check(lib().dco_server_submit(self._s, stream, _ptr(left), _ptr(right), _ptr(out), ctypes.byref(t)), None)
        self._keep[t.value] = (left, right, out)   # the buffers stay alive until the wait
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> RequestTimes:
        tm = RequestTimes()
        rc = lib().dco_server_wait(self._s, ticket, timeout_ms, ctypes.byref(tm))
        if rc != DCO_ETIMEOUT:
            self._keep.pop(ticket, None)
        _check(rc, None)
        return tm

    def counters(self) -> dict:
        b, f = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        mb, lb = c_size_t(), c_size_t()
        _check(lib().dco_server_counters(self._s, ctypes.byref(b), ctypes.byref(f), ctypes.byref(mb),
                                         ctypes.byref(lb)), None)
        return {"batches": b.value, "frames": f.value, "max_batch_bytes": mb.value, "lane_budget": lb.value}

    def close(self) -> None:
        if self._s:
            lib().dco_server_destroy(self._s)
            self._s = c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
