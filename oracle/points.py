"""FP64 CPU oracle of the point-cloud rasterizer and compositing: numpy
wrappers around ``points.c``.

TEST INFRASTRUCTURE ONLY.  The tests and the benchmark's CPU-baseline leg are
the only callers; the product package never imports this module, and this
module never imports the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "points.c")
_LIB_PATH = os.path.join(_HERE, "libpoints_oracle.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int

ALPHA = 0
NORM = 1

RIM = 1          # margin flags
DEPTH_TIE = 2
ZNEAR = 4
FWD_AMBIGUOUS = RIM | DEPTH_TIE | ZNEAR
GRAD_COND_AMBIGUOUS = RIM | ZNEAR


def build(force: bool = False) -> str:
    """Compile ``points.c`` into ``libpoints_oracle.so`` next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("ORACLE_POINTS_LIB") or build())
        L.orp_rasterize.argtypes = [_f64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64, _dbl, _i64p, _i64,
                                    _i64p, _f64p, _f64p]
        L.orp_margins.argtypes = [_f64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64, _dbl, _i64p, _i64, _dbl,
                                  _u8p]
        L.orp_composite_fwd.argtypes = [_i64, _i64, _i64p, _f64p, _f64p, _i64, _dbl, _int, _f64p]
        L.orp_composite_bwd.argtypes = [_i64, _i64, _i64p, _f64p, _f64p, _i64, _dbl, _int, _f64p, _f64p, _f64p,
                                        _f64p, _f64p]
        L.orp_rast_bwd.argtypes = [_f64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64, _i64p, _f64p, _f64p,
                                   _i64p, _i64, _f64p, _f64p]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a, t):
    return ctypes.cast(None, t) if a is None else a.ctypes.data_as(t)


class Clouds:
    """Packed point clouds: points (P,3), first_point/num_points (N,), cams (N,16); upcast to FP64."""

    def __init__(self, points, first_point, num_points, cams):
        self.points = _d(points).reshape(-1, 3)
        self.first = _i(first_point)
        self.num = _i(num_points)
        self.cams = _d(cams).reshape(-1, 16)

    @property
    def N(self):
        return int(self.first.shape[0])

    @property
    def P(self):
        return int(self.points.shape[0])

    @classmethod
    def from_batch(cls, b):
        g = (lambda k: b[k]) if isinstance(b, dict) else (lambda k: getattr(b, k))
        return cls(np.asarray(g("points"), np.float32), g("first_point"), g("num_points"),
                   np.asarray(g("cams"), np.float32))


def _pixels(pixels):
    if pixels is None:
        return None, 0
    px = _i(pixels).reshape(-1, 3)
    return px, px.shape[0]


def rasterize(c: Clouds, S, K, radius, pixels=None):
    """(idx (P,K) int64, zbuf (P,K), dists (P,K)) for the listed pixels (default: all)."""
    L = _load()
    px, npix = _pixels(pixels)
    if px is None:
        npix = c.N * S * S
    idx = np.empty((npix, K), np.int64)
    zb = np.empty((npix, K))
    di = np.empty((npix, K))
    L.orp_rasterize(_p(c.points, _f64p), c.P, _p(c.first, _i64p), _p(c.num, _i64p), c.N, _p(c.cams, _f64p),
                    S, K, float(radius), _p(px, _i64p), npix, _p(idx, _i64p), _p(zb, _f64p), _p(di, _f64p))
    return idx, zb, di


def margins(c: Clouds, S, K, radius, pixels=None, eps=1e-6):
    L = _load()
    px, npix = _pixels(pixels)
    if px is None:
        npix = c.N * S * S
    fl = np.zeros(npix, np.uint8)
    L.orp_margins(_p(c.points, _f64p), c.P, _p(c.first, _i64p), _p(c.num, _i64p), c.N, _p(c.cams, _f64p), S, K,
                  float(radius), _p(px, _i64p), npix, float(eps), _p(fl, _u8p))
    return fl


def composite_fwd(idx, dists, features, radius, mode=ALPHA):
    """(npix, D) composited features; idx/dists (..., K), features (P, D)."""
    L = _load()
    idx = _i(idx)
    K = idx.shape[-1]
    npix = idx.size // K
    feats = _d(features)
    D = feats.shape[-1]
    out = np.empty((npix, D))
    L.orp_composite_fwd(npix, K, _p(idx, _i64p), _p(_d(dists), _f64p), _p(feats, _f64p), D, float(radius), mode,
                        _p(out, _f64p))
    return out


def composite_bwd(idx, dists, features, radius, grad_out, mode=ALPHA, with_abs=False):
    """(grad_dists (npix, K), grad_features (P, D)[, grad_features_abs, grad_dists_abs]): the
    *_abs arrays hold the magnitudes of the terms that form each component."""
    L = _load()
    idx = _i(idx)
    K = idx.shape[-1]
    npix = idx.size // K
    feats = _d(features)
    D = feats.shape[-1]
    gdi = np.zeros((npix, K))
    gf = np.zeros_like(feats)
    ga = np.zeros_like(feats) if with_abs else None
    gda = np.zeros((npix, K)) if with_abs else None
    L.orp_composite_bwd(npix, K, _p(idx, _i64p), _p(_d(dists), _f64p), _p(feats, _f64p), D, float(radius), mode,
                        _p(_d(grad_out).reshape(npix, D), _f64p), _p(gdi, _f64p), _p(gf, _f64p), _p(ga, _f64p),
                        _p(gda, _f64p))
    return (gdi, gf, ga, gda) if with_abs else (gdi, gf)


def rast_bwd(c: Clouds, S, K, idx, grad_zbuf, grad_dists, pixels=None, with_abs=False):
    """dL/dpoints (P, 3) conditioned on idx[, magnitudes of the terms]."""
    L = _load()
    px, npix = _pixels(pixels)
    if px is None:
        npix = c.N * S * S
    gp = np.zeros_like(c.points)
    ga = np.zeros_like(c.points) if with_abs else None
    gz = None if grad_zbuf is None else _d(grad_zbuf).reshape(npix, K)
    gd = None if grad_dists is None else _d(grad_dists).reshape(npix, K)
    L.orp_rast_bwd(_p(c.points, _f64p), c.P, _p(c.first, _i64p), _p(c.num, _i64p), c.N, _p(c.cams, _f64p), S, K,
                   _p(_i(idx).reshape(npix, K), _i64p), _p(gz, _f64p), _p(gd, _f64p), _p(px, _i64p), npix,
                   _p(gp, _f64p), _p(ga, _f64p))
    return (gp, ga) if with_abs else gp
