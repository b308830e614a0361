"""FP64 CPU oracle of lit shading (flat, Gouraud, Phong) + softmax / hard
blending of mesh fragments: numpy wrappers around ``shading.c``.

TEST INFRASTRUCTURE ONLY.  The tests are the only callers; the product package
never imports this module, and this module never imports the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shading.c")
_LIB_PATH = os.path.join(_HERE, "libshading_oracle.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_int = ctypes.c_int

FLAT, GOURAUD, PHONG = 0, 1, 2
SOFTMAX, HARD = 0, 1


def build(force: bool = False) -> str:
    """Compile ``shading.c`` into ``libshading_oracle.so`` next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get("ORACLE_SHADING_LIB") or build())
        common = [_i64, _i64, _i64p, _i64p, _f64p, _f64p, _f64p, _i64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                  _int, _int]
        L.ors_shade_fwd.argtypes = common + [_f64p]
        L.ors_shade_bwd.argtypes = common + [_f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _i64, _f64p]
        L.ors_shade_margins.argtypes = [_i64, _i64, _i64p, _i64p, _f64p, _i64p, _f64p, _f64p, _f64p, _f64p, _int,
                                        _int, _f64p]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def light_params(position, ambient=(0.5, 0.5, 0.5), diffuse=(0.3, 0.3, 0.3), specular=(0.2, 0.2, 0.2),
                 shininess=64.0):
    return _d(list(position) + list(ambient) + list(diffuse) + list(specular) + [shininess])


def blend_params(sigma=1e-4, gamma=1e-4, znear=0.1, zfar=100.0, eps=1e-10, bg=(1.0, 1.0, 1.0)):
    return _d([sigma, gamma, znear, zfar, eps] + list(bg))


def _args(image, p2f, zbuf, bary, dists, faces, verts, normals, colors, cams, light, blend):
    p2f = _i(p2f)
    K = p2f.shape[-1]
    npix = p2f.size // K
    arrs = [_i(image).reshape(npix), p2f.reshape(npix, K), _d(zbuf).reshape(npix, K), _d(bary).reshape(npix, K, 3),
            _d(dists).reshape(npix, K), _i(faces).reshape(-1, 3), _d(verts).reshape(-1, 3),
            _d(normals).reshape(-1, 3), _d(colors).reshape(-1, 3), _d(cams).reshape(-1, 16), _d(light), _d(blend)]
    ptrs = [a.ctypes.data_as(_i64p if a.dtype == np.int64 else _f64p) for a in arrs]
    return npix, K, arrs, ptrs


def shade_fwd(image, p2f, zbuf, bary, dists, faces, verts, normals, colors, cams, light, blend, shading,
              blend_mode=SOFTMAX):
    """(npix, 4) RGBA; image[p] is the camera index of pixel p."""
    npix, K, arrs, ptrs = _args(image, p2f, zbuf, bary, dists, faces, verts, normals, colors, cams, light, blend)
    out = np.empty((npix, 4))
    _load().ors_shade_fwd(npix, K, *ptrs, shading, blend_mode, out.ctypes.data_as(_f64p))
    return out


def shade_bwd(image, p2f, zbuf, bary, dists, faces, verts, normals, colors, cams, light, blend, shading, grad_rgba,
              blend_mode=SOFTMAX, with_abs=False, with_abs_bary=False):
    """(grad_zbuf, grad_bary, grad_dists, grad_verts (direct), grad_normals, grad_colors[, abs][, abs_bary])
    where abs (3, V, 3) holds the magnitudes of the per-slot contributions to the last three and
    abs_bary (npix, K, 3) the magnitudes of the terms that form each grad_bary component."""
    npix, K, arrs, ptrs = _args(image, p2f, zbuf, bary, dists, faces, verts, normals, colors, cams, light, blend)
    V = arrs[6].shape[0]
    gz, gd = np.zeros((npix, K)), np.zeros((npix, K))
    gb = np.zeros((npix, K, 3))
    gv, gn, gc = np.zeros((V, 3)), np.zeros((V, 3)), np.zeros((V, 3))
    g = _d(grad_rgba).reshape(npix, 4)
    P = lambda a: a.ctypes.data_as(_f64p)
    ab = np.zeros((3, V, 3))
    abb = np.zeros((npix, K, 3))
    _load().ors_shade_bwd(npix, K, *ptrs, shading, blend_mode, P(g), P(gz), P(gb), P(gd), P(gv), P(gn), P(gc), P(ab),
                          V, P(abb))
    out = (gz, gb, gd, gv, gn, gc)
    if with_abs:
        out += (ab,)
    if with_abs_bary:
        out += (abb,)
    return out


def shade_margins(image, p2f, bary, faces, verts, normals, cams, light, shading, blend_mode=SOFTMAX):
    """Per pixel: the smallest |cos| (and |r . v| where lit) over the reflection evaluations
    the blend uses -- the distance to a kink of the reflection model."""
    p2f = _i(p2f)
    K = p2f.shape[-1]
    npix = p2f.size // K
    arrs = [_i(image).reshape(npix), p2f.reshape(npix, K), _d(bary).reshape(npix, K, 3), _i(faces).reshape(-1, 3),
            _d(verts).reshape(-1, 3), _d(normals).reshape(-1, 3), _d(cams).reshape(-1, 16), _d(light)]
    ptrs = [a.ctypes.data_as(_i64p if a.dtype == np.int64 else _f64p) for a in arrs]
    out = np.empty(npix)
    _load().ors_shade_margins(npix, K, *ptrs, shading, blend_mode, out.ctypes.data_as(_f64p))
    return out
