"""Brute-force CPU oracle for the exact running median (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA path and never imports the product
package.

Semantics (Section II, definition of the median element and of the running
median; Section III, proof of get_order_statistic): every output point takes
the window of n = 2r+1 pixels per axis centred on it, with coordinates clamped
to the image (replicate border, clamped pixels counted with multiplicity), and
returns the element of 0-based rank ``rank`` of the sorted window; the median
is rank (N-1)/2 with N = n**dims.

Two independent implementations live here:
  * ``median2d`` / ``median3d`` / ``points``: the C oracle (``hrm_oracle.c``),
    gather + qsort or gather + Quickselect per output point, threaded;
  * ``median2d_numpy`` / ``median3d_numpy``: the same definition written with
    numpy (edge padding + sliding windows + ``np.sort``), for small inputs.

Parity status: pinned (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hrm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

METHODS = {"sort": 0, "select": 1}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags: builds on x86_64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.oracle_filter2d.argtypes = [c.c_int, c.c_void_p, c.c_size_t, c.c_void_p, c.c_size_t,
                                        c.c_int, c.c_int, c.c_int, c.c_long, c.c_int, c.c_int]
        lib.oracle_filter3d.argtypes = [c.c_int, c.c_void_p, c.c_size_t, c.c_size_t,
                                        c.c_void_p, c.c_size_t, c.c_size_t,
                                        c.c_int, c.c_int, c.c_int, c.c_int, c.c_long, c.c_int, c.c_int]
        lib.oracle_points.argtypes = [c.c_int, c.c_void_p, c.c_size_t, c.c_size_t,
                                      c.c_int, c.c_int, c.c_int, c.c_int, c.c_int, c.c_long,
                                      c.c_void_p, c.c_void_p, c.c_void_p, c.c_long,
                                      c.c_void_p, c.c_int, c.c_int]
        for f in (lib.oracle_filter2d, lib.oracle_filter3d, lib.oracle_points):
            f.restype = c.c_int
        _lib = lib
    return _lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _check(img: np.ndarray, ndim: int) -> np.ndarray:
    if img.dtype not in (np.uint8, np.uint16):
        raise TypeError("oracle supports uint8 and uint16 only, got %s" % img.dtype)
    if img.ndim != ndim:
        raise ValueError("expected a %dD array" % ndim)
    return np.ascontiguousarray(img)


def _rank(rank, N):
    if rank is None:
        return -1
    if not 0 <= rank < N:
        raise ValueError("rank %d outside [0, %d)" % (rank, N))
    return int(rank)


def median2d(img: np.ndarray, r: int, rank: int | None = None, method: str = "select",
             threads: int | None = None) -> np.ndarray:
    """Exact 2D running order statistic (median by default) of a (H, W) image."""
    img = _check(img, 2)
    H, W = img.shape
    n = 2 * r + 1
    out = np.empty_like(img)
    rc = _load().oracle_filter2d(img.itemsize, img.ctypes.data, img.strides[0], out.ctypes.data,
                                 out.strides[0], W, H, r, _rank(rank, n * n), METHODS[method],
                                 threads or default_threads())
    if rc:
        raise RuntimeError("oracle_filter2d failed (%d)" % rc)
    return out


def median3d(vol: np.ndarray, r: int, rank: int | None = None, method: str = "select",
             threads: int | None = None) -> np.ndarray:
    """Exact 3D running order statistic with a cubic window of a (D, H, W) volume."""
    vol = _check(vol, 3)
    D, H, W = vol.shape
    n = 2 * r + 1
    out = np.empty_like(vol)
    rc = _load().oracle_filter3d(vol.itemsize, vol.ctypes.data, vol.strides[1], vol.strides[0],
                                 out.ctypes.data, out.strides[1], out.strides[0], W, H, D, r,
                                 _rank(rank, n ** 3), METHODS[method],
                                 threads or default_threads())
    if rc:
        raise RuntimeError("oracle_filter3d failed (%d)" % rc)
    return out


def points(img: np.ndarray, r: int, ys, xs, zs=None, rank: int | None = None,
           method: str = "select", threads: int | None = None) -> np.ndarray:
    """Filter outputs at selected points only.

    ``img`` is (H, W) for 2D (zs must be None) or (D, H, W) for 3D (cubic
    window, zs required).  Returns uint32 values in point order."""
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    if img.ndim == 2:
        if zs is not None:
            raise ValueError("zs given for a 2D image")
        img = _check(img, 2)
        H, W = img.shape
        D, rz, slice_ = 1, 0, 0
        zp = None
    else:
        img = _check(img, 3)
        D, H, W = img.shape
        rz, slice_ = r, img.strides[0]
        zs = np.ascontiguousarray(zs, dtype=np.int32)
        zp = zs.ctypes.data
    n = 2 * r + 1
    N = n * n * (2 * rz + 1)
    out = np.empty(len(xs), dtype=np.uint32)
    pitch = img.strides[-2]
    rc = _load().oracle_points(img.itemsize, img.ctypes.data, pitch, slice_, W, H, D, r, rz,
                               _rank(rank, N), xs.ctypes.data, ys.ctypes.data, zp, len(xs),
                               out.ctypes.data, METHODS[method], threads or default_threads())
    if rc:
        raise RuntimeError("oracle_points failed (%d)" % rc)
    return out


# ---- numpy restatement of the definition (small inputs only) -------------

def median2d_numpy(img: np.ndarray, r: int, rank: int | None = None) -> np.ndarray:
    """Definition written with numpy: pad by edge replication (= clamped
    coordinates), take every n x n window, sort it, pick the rank."""
    n = 2 * r + 1
    k = (n * n - 1) // 2 if rank is None else rank
    p = np.pad(img, r, mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(p, (n, n))
    flat = win.reshape(img.shape[0], img.shape[1], n * n)
    return np.sort(flat, axis=-1)[..., k].astype(img.dtype)


def median3d_numpy(vol: np.ndarray, r: int, rank: int | None = None) -> np.ndarray:
    n = 2 * r + 1
    k = (n ** 3 - 1) // 2 if rank is None else rank
    p = np.pad(vol, r, mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(p, (n, n, n))
    flat = win.reshape(vol.shape + (n ** 3,))
    return np.sort(flat, axis=-1)[..., k].astype(vol.dtype)
