"""ctypes wrapper of the FP64 C oracle (kf_oracle.c). Test infrastructure only.

Every function takes numpy arrays and returns numpy arrays; frames are uint8 [H, pitch]
or [T, H, pitch] with W <= pitch valid columns, maps are float64 [H, W].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_LIB = os.path.join(_HERE, "libkf_oracle.so")

HARRIS_K = 0.04
THRESHOLD = 1e-5
MAP_NAMES = ("f", "g1", "g", "ix", "iy", "pxx", "pxy", "pyy", "sxx", "sxy", "syy", "r")


def build(force: bool = False) -> str:
    """Compile kf_oracle.c into libkf_oracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.kfo_chain_frame.restype = i64
        L.kfo_chain_frame.argtypes = [i32, i32, vp, i64, dbl, dbl, vp, vp, i64]
        L.kfo_chain_volume.restype = i32
        L.kfo_chain_volume.argtypes = [i32, i32, i32, vp, i64, dbl, dbl, vp, vp, vp, i32]
        L.kfo_convert.argtypes = [i32, i32, vp, i64, vp]
        for f in ("kfo_gauss_h", "kfo_gauss_v", "kfo_box5"):
            getattr(L, f).argtypes = [i32, i32, vp, vp]
        L.kfo_sobel.argtypes = [i32, i32, vp, vp, vp]
        L.kfo_products.argtypes = [i64, vp, vp, vp, vp, vp]
        L.kfo_harris.argtypes = [i64, vp, vp, vp, dbl, vp]
        L.kfo_nms.restype = i64
        L.kfo_nms.argtypes = [i32, i32, vp, dbl, vp, i64]
        L.kfo_select_points.restype = i32
        L.kfo_select_points.argtypes = [i32, i32, vp, vp, i64, i32, vp]
        L.kfo_lk.argtypes = [i32, i32, vp, vp, vp, vp, i32, vp, i32, vp, vp, vp]
        L.kfo_track_pair.restype = i32
        L.kfo_track_pair.argtypes = [i32, i32, vp, vp, i64, dbl, dbl, i32, i32, vp, vp, vp, vp]
        L.kfo_track_volume.restype = i32
        L.kfo_track_volume.argtypes = [i32, i32, i32, vp, i64, dbl, dbl, i32, i32, vp, vp, vp, vp, vp, i32]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def convert(frame: np.ndarray, W: int | None = None) -> np.ndarray:
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    H, P = frame.shape
    W = P if W is None else W
    out = np.empty((H, W))
    lib().kfo_convert(H, W, _p(frame), P, _p(out))
    return out


def _map1(fn: str, m: np.ndarray) -> np.ndarray:
    m = _f64(m)
    out = np.empty_like(m)
    getattr(lib(), fn)(m.shape[0], m.shape[1], _p(m), _p(out))
    return out


def gauss_h(m): return _map1("kfo_gauss_h", m)
def gauss_v(m): return _map1("kfo_gauss_v", m)
def box5(m): return _map1("kfo_box5", m)


def sobel(g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    g = _f64(g)
    ix, iy = np.empty_like(g), np.empty_like(g)
    lib().kfo_sobel(g.shape[0], g.shape[1], _p(g), _p(ix), _p(iy))
    return ix, iy


def products(ix, iy):
    ix, iy = _f64(ix), _f64(iy)
    o = [np.empty_like(ix) for _ in range(3)]
    lib().kfo_products(ix.size, _p(ix), _p(iy), _p(o[0]), _p(o[1]), _p(o[2]))
    return tuple(o)


def harris(sxx, sxy, syy, k: float = HARRIS_K):
    sxx, sxy, syy = _f64(sxx), _f64(sxy), _f64(syy)
    r = np.empty_like(sxx)
    lib().kfo_harris(sxx.size, _p(sxx), _p(sxy), _p(syy), k, _p(r))
    return r


def nms(r: np.ndarray, thr: float = THRESHOLD) -> tuple[np.ndarray, int]:
    r = _f64(r)
    mask = np.empty(r.shape, dtype=np.uint8)
    c = lib().kfo_nms(r.shape[0], r.shape[1], _p(r), thr, _p(mask), r.shape[1])
    return mask, int(c)


def chain_frame(frame: np.ndarray, W: int | None = None, k: float = HARRIS_K,
                thr: float = THRESHOLD, want_maps: bool = True):
    """Whole chain on one frame [H, pitch]. Returns (maps dict or None, mask [H, W], count)."""
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    H, P = frame.shape
    W = P if W is None else W
    maps = {n: np.empty((H, W)) for n in MAP_NAMES} if want_maps else None
    ptrs = (ctypes.c_void_p * len(MAP_NAMES))(*[_p(maps[n]) for n in MAP_NAMES]) if want_maps \
        else None
    mask = np.empty((H, W), dtype=np.uint8)
    c = lib().kfo_chain_frame(H, W, _p(frame), P, k, thr,
                              ctypes.cast(ptrs, ctypes.c_void_p) if ptrs is not None else None,
                              _p(mask), W)
    if c < 0:
        raise MemoryError("oracle allocation failed")
    return maps, mask, int(c)


def chain_volume(frames: np.ndarray, W: int | None = None, k: float = HARRIS_K,
                 thr: float = THRESHOLD, want_r: bool = False, nthreads: int = 0):
    """Chain over frames [T, H, pitch] on all host cores (OpenMP over frames).

    Returns (masks [T, H, pitch] uint8 (columns >= W untouched = 0), counts [T] int32,
    r [T, H, W] float64 or None, threads used)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, P = frames.shape
    W = P if W is None else W
    masks = np.zeros_like(frames)
    counts = np.zeros(T, dtype=np.int32)
    r = np.empty((T, H, W)) if want_r else None
    used = lib().kfo_chain_volume(T, H, W, _p(frames), P, k, thr, _p(masks), _p(counts),
                                  _p(r) if r is not None else None, nthreads)
    return masks, counts, r, int(used)


def select_points(r: np.ndarray, mask: np.ndarray, K: int = 256) -> np.ndarray:
    r = _f64(r)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    idx = np.empty(K, dtype=np.int32)
    n = lib().kfo_select_points(r.shape[0], r.shape[1], _p(r), _p(mask), mask.shape[1], K,
                                _p(idx))
    return idx[:n].copy()


def lk(g_prev, g_cur, ix, iy, idx, win: int = 3):
    g_prev, g_cur, ix, iy = _f64(g_prev), _f64(g_cur), _f64(ix), _f64(iy)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = idx.size
    u, v = np.empty(n), np.empty(n)
    st = np.empty(n, dtype=np.int32)
    lib().kfo_lk(g_prev.shape[0], g_prev.shape[1], _p(g_prev), _p(g_cur), _p(ix), _p(iy), n,
                 _p(idx), win, _p(u), _p(v), _p(st))
    return u, v, st


def track_pair(prev: np.ndarray, cur: np.ndarray, W: int | None = None, K: int = 256,
               win: int = 3, k: float = HARRIS_K, thr: float = THRESHOLD):
    """LK tracking of the corners of `cur` against `prev` (frames [H, pitch]).

    Returns (idx [n] raster indices, u [n], v [n], status [n])."""
    prev = np.ascontiguousarray(prev, dtype=np.uint8)
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    H, P = cur.shape
    W = P if W is None else W
    idx = np.empty(K, dtype=np.int32)
    u, v = np.empty(K), np.empty(K)
    st = np.empty(K, dtype=np.int32)
    n = lib().kfo_track_pair(H, W, _p(prev), _p(cur), P, k, thr, K, win, _p(idx), _p(u), _p(v),
                             _p(st))
    if n < 0:
        raise MemoryError("oracle allocation failed")
    return idx[:n].copy(), u[:n].copy(), v[:n].copy(), st[:n].copy()


def track_volume(frames: np.ndarray, W: int | None = None, K: int = 256, win: int = 3, k: float = HARRIS_K,
                 thr: float = THRESHOLD, nthreads: int = 0):
    """Tracking of every frame pair of frames [T, H, pitch] on all host cores.

    Returns (n [T], idx [T, K], u [T, K], v [T, K], status [T, K], threads used)."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, P = frames.shape
    W = P if W is None else W
    n = np.zeros(T, dtype=np.int32)
    idx = np.full((T, K), -1, dtype=np.int32)
    u, v = np.zeros((T, K)), np.zeros((T, K))
    st = np.zeros((T, K), dtype=np.int32)
    used = lib().kfo_track_volume(T, H, W, _p(frames), P, k, thr, K, win, _p(n), _p(idx), _p(u), _p(v), _p(st),
                                  nthreads)
    if T > 1 and int(n[1:].min()) < 0:
        raise MemoryError("oracle allocation failed")
    return n, idx, u, v, st, int(used)
