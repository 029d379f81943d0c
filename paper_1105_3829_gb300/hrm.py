"""Thin ctypes binding of libhrm (include/hrm.h).

Only argument marshalling lives here: every filter step runs in the CUDA
kernels of libhrm.so.  There is no CPU fallback; if the library has not been
built, ``lib()`` raises.  Two layers are offered:

* ``hrm_*`` functions with the C names and signatures (pointers as ints,
  pitches in bytes, stream as a cudaStream_t handle int);
* tensor helpers (``filter2d``, ``filter3d``, ``rank_filter2d`` ...) that take
  torch CUDA tensors of dtype uint8 / uint16 and use torch only for device
  memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# HRM_LIB_VARIANT=count loads the instrumented build (_build/count/libhrm.so).
_VARIANT = os.environ.get("HRM_LIB_VARIANT", "")
LIB_PATH = os.path.join(PKG, "_build", _VARIANT, "libhrm.so") if _VARIANT else os.path.join(PKG, "_build", "libhrm.so")

HRM_U8, HRM_U16 = 1, 2
HRM_BORDER_REPLICATE = 0
HRM_ADAPTIVE = 1
HRM_MAX_RADIUS_2D = 127
HRM_MAX_RADIUS_3D = 19

STATUS = {0: "HRM_OK", 1: "HRM_EAGAIN", -1: "HRM_EINVAL", -2: "HRM_ENOMEM", -3: "HRM_ECUDA",
          -4: "HRM_ETIMEDOUT", -5: "HRM_ECANCELED", -6: "HRM_ENOTSUP", -7: "HRM_EDEVICE"}
HRM_OK, HRM_EAGAIN, HRM_EINVAL, HRM_ENOMEM, HRM_ECUDA = 0, 1, -1, -2, -3
HRM_ETIMEDOUT, HRM_ECANCELED, HRM_ENOTSUP, HRM_EDEVICE = -4, -5, -6, -7


class HRMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class hrm_job(C.Structure):
    _fields_ = [("dtype", C.c_int), ("dims", C.c_int), ("src", C.c_void_p), ("src_pitch", C.c_size_t),
                ("src_slice_pitch", C.c_size_t), ("dst", C.c_void_p), ("dst_pitch", C.c_size_t),
                ("dst_slice_pitch", C.c_size_t), ("width", C.c_int), ("height", C.c_int),
                ("depth", C.c_int), ("radius", C.c_int), ("rank", C.c_long), ("flags", C.c_uint),
                ("topo", C.c_void_p)]


class hrm_plan(C.Structure):
    _fields_ = [("tile_width", C.c_int), ("strip_height", C.c_int), ("slot_kbytes", C.c_int),
                ("path", C.c_int), ("tree", C.c_int)]


class hrm_request(C.Structure):
    _fields_ = [("dtype", C.c_int), ("width", C.c_int), ("height", C.c_int), ("radius", C.c_int),
                ("flags", C.c_uint), ("src", C.c_void_p), ("src_pitch", C.c_size_t),
                ("dst", C.c_void_p), ("dst_pitch", C.c_size_t), ("src_on_host", C.c_int),
                ("dst_on_host", C.c_int), ("topo", C.c_void_p)]


class hrm_topology_info(C.Structure):
    _fields_ = [("dtype", C.c_int), ("mode", C.c_uint), ("vmin", C.c_uint), ("vmax", C.c_uint),
                ("edge", C.c_uint * 17)]


class hrm_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64), ("waves", C.c_uint64), ("bytes_resident", C.c_uint64),
                ("bytes_high_water", C.c_uint64), ("arena_bytes", C.c_uint64), ("inflight", C.c_int),
                ("queued", C.c_int)]


_P, _S, _I, _U, _L = C.c_void_p, C.c_size_t, C.c_int, C.c_uint, C.c_long
SIGNATURES = {
    "hrm_version": (_I, []),
    "hrm_last_error": (C.c_char_p, []),
    "hrm_device_status": (_I, [_P]),
    "hrm_filter2d": (_I, [_I, _P, _S, _P, _S, _I, _I, _I, _I, _U, _P]),
    "hrm_filter3d": (_I, [_I, _P, _S, _S, _P, _S, _S, _I, _I, _I, _I, _I, _U, _P]),
    "hrm_rank_filter2d": (_I, [_I, _P, _S, _P, _S, _I, _I, _I, _L, _I, _U, _P]),
    "hrm_rank_filter3d": (_I, [_I, _P, _S, _S, _P, _S, _S, _I, _I, _I, _I, _L, _I, _U, _P]),
    "hrm_filter2d_lowprec": (_I, [_I, _P, _S, _P, _S, _I, _I, _I, _I, _P]),
    "hrm_topology_create": (_I, [C.POINTER(_P)]),
    "hrm_topology_destroy": (_I, [_P]),
    "hrm_filter2d_video": (_I, [_I, _P, _S, _P, _S, _I, _I, _I, _P, _P]),
    "hrm_topology_get": (_I, [_P, _P, C.POINTER(hrm_topology_info)]),
    "hrm_filter_batch": (_I, [C.POINTER(hrm_job), _I, _P]),
    "hrm_filter_batch_noalloc": (_I, [C.POINTER(hrm_job), _I, _P]),
    "hrm_batch_graph_create": (_I, [C.POINTER(hrm_job), _I, _P, C.POINTER(_P)]),
    "hrm_batch_graph_launch": (_I, [_P, _P]),
    "hrm_batch_graph_status": (_I, [_P, _P]),
    "hrm_batch_graph_destroy": (_I, [_P]),
    "hrm_autotune": (_I, [_I, _I, _I, _I, _I, _I, _U, _P, _S, _S, _P, C.POINTER(hrm_plan)]),
    "hrm_get_plan": (_I, [_I, _I, _I, _I, _I, _I, _U, C.POINTER(hrm_plan)]),
    "hrm_set_plan": (_I, [_I, _I, _I, _I, _I, _I, _U, C.POINTER(hrm_plan)]),
    "hrm_plan_save": (_I, [C.c_char_p]),
    "hrm_plan_load": (_I, [C.c_char_p]),
    "hrm_server_create": (_I, [_P, _S, _I, _I, C.POINTER(_P)]),
    "hrm_submit": (_I, [_P, C.POINTER(hrm_request), C.POINTER(C.c_uint64)]),
    "hrm_poll": (_I, [_P, C.c_uint64, _I]),
    "hrm_ticket_latency_us": (C.c_double, [_P, C.c_uint64]),
    "hrm_server_stats_get": (_I, [_P, C.POINTER(hrm_server_stats)]),
    "hrm_server_destroy": (_I, [_P]),
    # test hook (not in include/hrm.h): plant a device error code from the host
    "hrm_debug_set_error_word": (_I, [_I, _P, _U]),
}

_lib = None


def lib():
    """Load libhrm.so (built in-tree by paper_1105_3829_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhrm.so is not built (%s); run paper_1105_3829_gb300.build.build() "
                               "or __graft_entry__.build() first" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().hrm_last_error().decode(errors="replace")


def check(rc: int, what: str = "") -> int:
    if rc < 0:
        raise HRMError(rc, "%s: %s" % (what, last_error()))
    return rc


# ---- C-name mirrors -----------------------------------------------------------

def _fwd(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = "Direct call of the C entry point %s (see include/hrm.h)." % name
    return f


for _n in SIGNATURES:
    globals()[_n] = _fwd(_n)


# ---- tensor helpers -------------------------------------------------------------

def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.uint8:
        return HRM_U8
    if t.dtype == torch.uint16:
        return HRM_U16
    raise TypeError("expected a uint8 or uint16 tensor, got %s" % t.dtype)


def _stream(stream):
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check_img(t, ndim):
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if t.dim() != ndim:
        raise ValueError("expected a %dD tensor" % ndim)
    if t.stride(-1) != 1:
        raise ValueError("innermost dimension must be contiguous")


def filter2d(img, radius: int, adaptive: bool = False, out=None, stream=None):
    """Exact 2D median (replicate border) of a (H, W) uint8/uint16 CUDA tensor."""
    _check_img(img, 2)
    out = _torch().empty_like(img) if out is None else out
    _check_img(out, 2)
    es = img.element_size()
    rc = lib().hrm_filter2d(_dtype_code(img), img.data_ptr(), img.stride(0) * es, out.data_ptr(),
                            out.stride(0) * es, img.shape[1], img.shape[0], radius,
                            HRM_BORDER_REPLICATE, HRM_ADAPTIVE if adaptive else 0, _stream(stream))
    check(rc, "hrm_filter2d")
    return out


def rank_filter2d(img, radius: int, rank: int, adaptive: bool = False, out=None, stream=None):
    """Exact 2D order statistic of 0-based rank ``rank`` of every window."""
    _check_img(img, 2)
    out = _torch().empty_like(img) if out is None else out
    es = img.element_size()
    rc = lib().hrm_rank_filter2d(_dtype_code(img), img.data_ptr(), img.stride(0) * es, out.data_ptr(),
                                 out.stride(0) * es, img.shape[1], img.shape[0], radius, rank,
                                 HRM_BORDER_REPLICATE, HRM_ADAPTIVE if adaptive else 0, _stream(stream))
    check(rc, "hrm_rank_filter2d")
    return out


def filter2d_lowprec(img, radius: int, drop_bits: int, out=None, stream=None):
    """Reduced-precision median: exact median with its drop_bits lowest bits cleared."""
    _check_img(img, 2)
    out = _torch().empty_like(img) if out is None else out
    es = img.element_size()
    rc = lib().hrm_filter2d_lowprec(_dtype_code(img), img.data_ptr(), img.stride(0) * es, out.data_ptr(),
                                    out.stride(0) * es, img.shape[1], img.shape[0], radius, drop_bits,
                                    _stream(stream))
    check(rc, "hrm_filter2d_lowprec")
    return out


def filter3d(vol, radius: int, adaptive: bool = False, out=None, stream=None, rank: int | None = None):
    """Exact 3D median (cubic window) of a (D, H, W) uint8/uint16 CUDA tensor."""
    _check_img(vol, 3)
    out = _torch().empty_like(vol) if out is None else out
    _check_img(out, 3)
    es = vol.element_size()
    args = (_dtype_code(vol), vol.data_ptr(), vol.stride(1) * es, vol.stride(0) * es, out.data_ptr(),
            out.stride(1) * es, out.stride(0) * es, vol.shape[2], vol.shape[1], vol.shape[0], radius)
    flags = HRM_ADAPTIVE if adaptive else 0
    if rank is None:
        rc = lib().hrm_filter3d(*args, HRM_BORDER_REPLICATE, flags, _stream(stream))
    else:
        rc = lib().hrm_rank_filter3d(*args, rank, HRM_BORDER_REPLICATE, flags, _stream(stream))
    check(rc, "hrm_filter3d")
    return out


def make_job(src, dst, radius: int, rank: int = -1, adaptive: bool = False, topo=None) -> hrm_job:
    """Batch job descriptor for a (H, W) or (D, H, W) tensor pair; ``topo``
    (a Topology) makes the job one frame of that stream."""
    es = src.element_size()
    j = hrm_job()
    j.dtype = _dtype_code(src)
    j.dims = src.dim()
    j.src, j.dst = src.data_ptr(), dst.data_ptr()
    j.src_pitch, j.dst_pitch = src.stride(-2) * es, dst.stride(-2) * es
    if src.dim() == 3:
        j.src_slice_pitch, j.dst_slice_pitch = src.stride(0) * es, dst.stride(0) * es
        j.depth = src.shape[0]
    else:
        j.depth = 1
    j.width, j.height = src.shape[-1], src.shape[-2]
    j.radius, j.rank, j.flags = radius, rank, HRM_ADAPTIVE if adaptive else 0
    j.topo = topo._h.value if topo is not None else None
    return j


def filter_batch(jobs, stream=None) -> None:
    arr = (hrm_job * len(jobs))(*jobs)
    check(lib().hrm_filter_batch(arr, len(jobs), _stream(stream)), "hrm_filter_batch")


def filter_batch_noalloc(jobs, stream=None) -> None:
    """hrm_filter_batch_noalloc: the batched filter without any device
    allocation (at most 64 jobs per call; see include/hrm.h)."""
    arr = (hrm_job * len(jobs))(*jobs)
    check(lib().hrm_filter_batch_noalloc(arr, len(jobs), _stream(stream)), "hrm_filter_batch_noalloc")


class BatchGraph:
    """A captured batched launch for a fixed job list (CUDA graph replay)."""

    def __init__(self, jobs, stream=None):
        self._jobs = (hrm_job * len(jobs))(*jobs)
        h = C.c_void_p()
        check(lib().hrm_batch_graph_create(self._jobs, len(jobs), _stream(stream), C.byref(h)),
              "hrm_batch_graph_create")
        self._h = h

    def launch(self, stream=None):
        check(lib().hrm_batch_graph_launch(self._h, _stream(stream)), "hrm_batch_graph_launch")

    def status(self, stream=None) -> int:
        """hrm_batch_graph_status: wait for the stream, raise on a kernel error flag of this graph."""
        return check(lib().hrm_batch_graph_status(self._h, _stream(stream)), "hrm_batch_graph_status")

    def close(self):
        if self._h:
            lib().hrm_batch_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_status(stream=None) -> int:
    return check(lib().hrm_device_status(_stream(stream)), "hrm_device_status")


def autotune(img, radius: int, adaptive: bool = False, stream=None) -> hrm_plan:
    """Time candidate plans on ``img`` (a (H, W) or (D, H, W) CUDA tensor) and
    cache the fastest for this problem class; returns it."""
    p = hrm_plan()
    es = img.element_size()
    dims = img.dim()
    W, H = img.shape[-1], img.shape[-2]
    D = img.shape[0] if dims == 3 else 1
    check(lib().hrm_autotune(_dtype_code(img), dims, W, H, D, radius, HRM_ADAPTIVE if adaptive else 0,
                             img.data_ptr(), img.stride(-2) * es, img.stride(0) * es if dims == 3 else 0,
                             _stream(stream), C.byref(p)), "hrm_autotune")
    return p


def get_plan(dtype: int, dims: int, width: int, height: int, depth: int, radius: int,
             adaptive: bool = False) -> hrm_plan:
    p = hrm_plan()
    check(lib().hrm_get_plan(dtype, dims, width, height, depth, radius, HRM_ADAPTIVE if adaptive else 0,
                             C.byref(p)), "hrm_get_plan")
    return p


def set_plan(dtype: int, dims: int, width: int, height: int, depth: int, radius: int, plan: hrm_plan,
             adaptive: bool = False) -> None:
    check(lib().hrm_set_plan(dtype, dims, width, height, depth, radius, HRM_ADAPTIVE if adaptive else 0,
                             C.byref(plan)), "hrm_set_plan")


class Topology:
    """Frame-to-frame median estimate for hrm_filter2d_video (device state)."""

    def __init__(self):
        h = _P()
        check(lib().hrm_topology_create(C.byref(h)), "hrm_topology_create")
        self._h = h

    def info(self, stream=None) -> dict:
        """The top level the next frame will use (waits for ``stream``)."""
        i = hrm_topology_info()
        check(lib().hrm_topology_get(self._h, _stream(stream), C.byref(i)), "hrm_topology_get")
        return {"dtype": i.dtype, "mode": i.mode, "vmin": i.vmin, "vmax": i.vmax, "edge": list(i.edge)}

    def close(self) -> None:
        if self._h:
            lib().hrm_topology_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filter2d_video(img, radius: int, topo: Topology, out=None, stream=None):
    """Exact 2D median of one frame of a stream; the top level of the tree
    comes from the previous frame's output held by ``topo``."""
    _check_img(img, 2)
    out = _torch().empty_like(img) if out is None else out
    es = img.element_size()
    rc = lib().hrm_filter2d_video(_dtype_code(img), img.data_ptr(), img.stride(0) * es, out.data_ptr(),
                                  out.stride(0) * es, img.shape[1], img.shape[0], radius, topo._h,
                                  _stream(stream))
    check(rc, "hrm_filter2d_video")
    return out


class Server:
    """Continuous-batching serving loop over a caller-provided device arena."""

    def __init__(self, arena, max_inflight: int = 256, max_queue: int = 0):
        self.arena = arena  # keep the tensor alive
        h = C.c_void_p()
        check(lib().hrm_server_create(arena.data_ptr(), arena.numel() * arena.element_size(), max_inflight,
                                      max_queue, C.byref(h)), "hrm_server_create")
        self._h = h

    def submit(self, src, dst, radius: int, adaptive: bool = False, topo=None) -> int:
        """Queue one 2D request; src/dst are torch tensors (CUDA or pinned CPU);
        ``topo`` (a Topology) makes it the next frame of that stream.
        Returns the ticket, or raises HRMError (code HRM_EAGAIN when the queue is full)."""
        q = hrm_request()
        q.dtype = _dtype_code(src)
        q.height, q.width = src.shape
        q.radius, q.flags = radius, HRM_ADAPTIVE if adaptive else 0
        es = src.element_size()
        q.src, q.src_pitch, q.src_on_host = src.data_ptr(), src.stride(0) * es, int(not src.is_cuda)
        q.dst, q.dst_pitch, q.dst_on_host = dst.data_ptr(), dst.stride(0) * es, int(not dst.is_cuda)
        q.topo = topo._h.value if topo is not None else None
        t = C.c_uint64()
        rc = lib().hrm_submit(self._h, C.byref(q), C.byref(t))
        if rc != HRM_OK:
            raise HRMError(rc, "hrm_submit: %s" % last_error())
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0) -> int:
        return lib().hrm_poll(self._h, ticket, timeout_us)

    def latency_us(self, ticket: int) -> float:
        return lib().hrm_ticket_latency_us(self._h, ticket)

    def stats(self) -> hrm_server_stats:
        s = hrm_server_stats()
        check(lib().hrm_server_stats_get(self._h, C.byref(s)), "hrm_server_stats_get")
        return s

    def close(self):
        if self._h:
            lib().hrm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
