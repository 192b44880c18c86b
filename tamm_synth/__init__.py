"""Seeded synthetic inputs shared by the FP64 oracle and the GPU library's tests/bench.

Holds no contraction arithmetic: it draws Philox4x32-10 / Box-Muller normals per
dense element and antisymmetrises same-space mode pairs (see ``synth.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libtamm_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libtamm_synth.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.tamm_synth_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            lib.tamm_synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
            lib.tamm_synth_normal.restype = ctypes.c_double
            lib.tamm_synth_value.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                             i64p, ctypes.c_int, ctypes.c_int, i64p]
            lib.tamm_synth_value.restype = ctypes.c_double
            lib.tamm_synth_fill_boxes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int,
                                                  i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, i64p, i64p, i64p,
                                                  ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def philox4x32_10(ctr, key) -> tuple:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.tamm_synth_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def normal(seed: int, stream: int, index: int) -> float:
    return _load().tamm_synth_normal(seed, stream, index)


def value(seed: int, stream: int, sigma: float, dims, anti01: bool, anti23: bool, idx) -> float:
    d = _i64(dims)
    i = _i64(idx)
    return _load().tamm_synth_value(seed, stream, sigma, len(d), _p64(d), int(anti01), int(anti23), _p64(i))


def fill_boxes(seed: int, stream: int, sigma: float, dims, anti01: bool, anti23: bool,
               lo, ext, off, out: np.ndarray, sym01: bool = False) -> None:
    """Fill boxes ``[lo[b], lo[b]+ext[b])`` of a dense tensor, row-major, at ``out[off[b]:]``.

    ``sym01`` symmetrises modes 0 and 1 of a 3-mode tensor instead (Cholesky vectors)."""
    lo = _i64(lo).reshape(-1, len(dims))
    ext = _i64(ext).reshape(-1, len(dims))
    off = _i64(off).reshape(-1)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    nbox = lo.shape[0]
    assert ext.shape[0] == nbox and off.shape[0] == nbox
    if nbox:
        need = int((off + ext.prod(axis=1)).max())
        assert need <= out.size, (need, out.size)
    d = _i64(dims)
    pair01 = int(anti01)
    if sym01:
        assert len(d) == 3 and d[0] == d[1] and not anti01, "sym01: 3-mode tensors with equal first two extents"
        pair01 = 2
    _load().tamm_synth_fill_boxes(seed, stream, sigma, len(d), _p64(d), pair01, int(anti23), nbox,
                                  _p64(lo), _p64(ext), _p64(off),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
