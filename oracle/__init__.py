"""FP64 CPU oracle: numpy wrappers around ``oracle.c``.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers; the product package never
imports this module, and this module never imports the product package.

Every function takes the packed-batch arrays (any float dtype is upcast to
float64 before the call) and returns float64 / int64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, no FMA contraction),
    and the point-cloud (``points.c``), shading (``shading.c``) and nearest-neighbour
    (``knn.c``) oracles beside it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    from . import knn, points, shading
    points.build(force)
    shading.build(force)
    knn.build(force)
    return _LIB_PATH


def _open(path):
    L = ctypes.CDLL(path)
    L.orc_rasterize.argtypes = [_f64p, _i64, _i64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64,
                                _dbl, _int, _int, _i64p, _i64, _i64p, _f64p, _f64p, _f64p]
    L.orc_pixel_candidates.argtypes = [_f64p, _i64, _i64p, _i64, _i64p, _i64p, _f64p, _i64, _dbl,
                                       _int, _int, _i64, _i64, _i64, _i64p, _f64p, _i64]
    L.orc_pixel_candidates.restype = _i64
    L.orc_margins.argtypes = [_f64p, _i64, _i64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64,
                              _dbl, _int, _int, _i64p, _i64, _dbl, _u8p]
    L.orc_bins.argtypes = [_f64p, _i64, _i64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64, _dbl,
                           _dbl, _i64p, _i64p, _i64p, _u8p]
    L.orc_blend_fwd.argtypes = [_i64, _i64, _i64p, _f64p, _f64p, _f64p, _i64p, _f64p, _dbl, _dbl,
                                _dbl, _dbl, _f64p, _int, _dbl, _f64p]
    L.orc_blend_bwd.argtypes = [_i64, _i64, _i64p, _f64p, _f64p, _f64p, _i64p, _f64p, _dbl, _dbl,
                                _dbl, _dbl, _f64p, _int, _dbl, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.orc_rast_bwd.argtypes = [_f64p, _i64, _i64p, _i64, _i64p, _i64p, _i64, _f64p, _i64, _i64,
                               _dbl, _int, _int, _i64p, _i64, _i64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    return L


def _load():
    # ORACLE_MESH_LIB names another build of oracle.c: the mutation tests plant
    # a mistake in a copy of the source and check that the pins fail
    global _lib
    if _lib is None:
        _lib = _open(os.environ.get("ORACLE_MESH_LIB") or build())
    return _lib


def compile_source(src_text, out_path):
    """Compile C source text of the oracle into a shared library at out_path."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o",
                           out_path, c_path, "-lm"])
    return out_path


def source_text():
    with open(_SRC) as f:
        return f.read()


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _p(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


class Mesh:
    """Packed batch, upcast to FP64 once."""

    def __init__(self, verts, faces, first_face, num_faces, cams):
        self.verts = _d(verts).reshape(-1, 3)
        self.faces = _i(faces).reshape(-1, 3)
        self.first_face = _i(first_face).reshape(-1)
        self.num_faces = _i(num_faces).reshape(-1)
        self.cams = _d(cams).reshape(-1, 16)

    @classmethod
    def from_batch(cls, b):
        return cls(b.verts, b.faces, b.first_face, b.num_faces, b.cams)

    @property
    def N(self):
        return self.first_face.shape[0]

    def _head(self):
        return (_p(self.verts, _f64p), self.verts.shape[0], _p(self.faces, _i64p), self.faces.shape[0],
                _p(self.first_face, _i64p), _p(self.num_faces, _i64p))


def _pixels(pixels):
    if pixels is None:
        return None, 0
    px = _i(pixels).reshape(-1, 3)
    return px, px.shape[0]


def rasterize(m: Mesh, S, K, blur=0.0, persp=True, clip=False, pixels=None):
    """K nearest fragments by brute force.  Returns (pix_to_face, zbuf, bary, dists)
    shaped (P, K), (P, K), (P, K, 3), (P, K); P = N*S*S when ``pixels`` is None."""
    L = _load()
    px, P = _pixels(pixels)
    if px is None:
        P = m.N * S * S
    p2f = np.empty((P, K), np.int64)
    zb = np.empty((P, K), np.float64)
    ba = np.empty((P, K, 3), np.float64)
    di = np.empty((P, K), np.float64)
    V, = m.verts.shape[:1]
    L.orc_rasterize(*m._head(), m.N, _p(m.cams, _f64p), S, K, float(blur), int(persp), int(clip),
                    _p(px, _i64p), P, _p(p2f, _i64p), _p(zb, _f64p), _p(ba, _f64p), _p(di, _f64p))
    return p2f, zb, ba, di


def candidates(m: Mesh, S, n, r, c, blur=0.0, persp=True, clip=False):
    """All candidate faces at pixel (n, r, c), sorted by (z, face id); returns (faces, z)."""
    L = _load()
    cap = m.faces.shape[0] + 1
    fo = np.empty(cap, np.int64)
    zo = np.empty(cap, np.float64)
    cnt = L.orc_pixel_candidates(*m._head(), _p(m.cams, _f64p), S, float(blur), int(persp), int(clip),
                                 n, r, c, _p(fo, _i64p), _p(zo, _f64p), cap)
    return fo[:cnt].copy(), zo[:cnt].copy()


def margins(m: Mesh, S, K, blur=0.0, persp=True, clip=False, pixels=None, eps=1e-6):
    """Per-pixel ambiguity bits (see ``orc_margins``)."""
    L = _load()
    px, P = _pixels(pixels)
    if px is None:
        P = m.N * S * S
    fl = np.zeros(P, np.uint8)
    L.orc_margins(*m._head(), m.N, _p(m.cams, _f64p), S, K, float(blur), int(persp), int(clip),
                  _p(px, _i64p), P, float(eps), _p(fl, _u8p))
    return fl


FWD_AMBIGUOUS = 1 | 2 | 4 | 8 | 16 | 128
GRAD_AMBIGUOUS = FWD_AMBIGUOUS | 32 | 64
# for gradients conditioned on a given face selection: depth ties (8) and the
# blur boundary (2) decide which faces are selected, not the adjoint of a slot
GRAD_COND_AMBIGUOUS = GRAD_AMBIGUOUS & ~(2 | 8)


def bins(m: Mesh, S, bin_size, blur=0.0, eps=1e-6):
    """Bin lists: returns (counts (N,nb,nb), offsets (N*nb*nb+1,), lists, amb)."""
    L = _load()
    nb = (S + bin_size - 1) // bin_size
    counts = np.zeros(m.N * nb * nb, np.int64)
    L.orc_bins(*m._head(), m.N, _p(m.cams, _f64p), S, bin_size, float(blur), float(eps),
               _p(counts, _i64p), None, None, None)
    offs = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    lists = np.zeros(int(offs[-1]), np.int64)
    amb = np.zeros(int(offs[-1]), np.uint8)
    L.orc_bins(*m._head(), m.N, _p(m.cams, _f64p), S, bin_size, float(blur), float(eps),
               _p(counts, _i64p), _p(offs, _i64p), _p(lists, _i64p), _p(amb, _u8p))
    return counts.reshape(m.N, nb, nb), offs, lists, amb


def blend_fwd(pix_to_face, zbuf, bary, dists, faces, colors, sigma, gamma, znear, zfar,
              bg=(1.0, 1.0, 1.0), mode=1, eps=1e-10):
    """Algorithm 1 (+ Algorithm 2 when mode == 1).  Inputs shaped (..., K); returns (..., 4)."""
    L = _load()
    p2f = _i(pix_to_face)
    K = p2f.shape[-1]
    lead = p2f.shape[:-1]
    P = int(np.prod(lead)) if lead else 1
    zb, ba, di = _d(zbuf), _d(bary), _d(dists)
    fa = _i(faces).reshape(-1, 3) if faces is not None else np.zeros((1, 3), np.int64)
    co = _d(colors).reshape(-1, 3) if colors is not None else np.zeros((1, 3))
    bgv = _d(bg)
    out = np.empty((P, 4), np.float64)
    L.orc_blend_fwd(P, K, _p(p2f, _i64p), _p(zb, _f64p), _p(ba, _f64p), _p(di, _f64p), _p(fa, _i64p),
                    _p(co, _f64p), sigma, gamma, znear, zfar, _p(bgv, _f64p), int(mode), eps,
                    _p(out, _f64p))
    return out.reshape(*lead, 4)


def blend_bwd(pix_to_face, zbuf, bary, dists, faces, colors, grad_rgba, sigma, gamma, znear, zfar,
              bg=(1.0, 1.0, 1.0), mode=1, eps=1e-10, V=None, with_abs=False):
    """Adjoint of ``blend_fwd``: returns (grad_zbuf, grad_bary, grad_dists, grad_colors).  With
    ``with_abs`` also the per-component sums of |contribution| to grad_colors and the per-slot
    absolute-term scales (grad_zbuf_abs, grad_bary_abs, grad_dists_abs)."""
    L = _load()
    p2f = _i(pix_to_face)
    K = p2f.shape[-1]
    lead = p2f.shape[:-1]
    P = int(np.prod(lead)) if lead else 1
    zb, ba, di = _d(zbuf), _d(bary), _d(dists)
    fa = _i(faces).reshape(-1, 3) if faces is not None else np.zeros((1, 3), np.int64)
    co = _d(colors).reshape(-1, 3) if colors is not None else np.zeros((1, 3))
    g = _d(grad_rgba)
    bgv = _d(bg)
    gz = np.empty((P, K)); gb = np.empty((P, K, 3)); gd = np.empty((P, K))
    gc = np.zeros((co.shape[0] if V is None else V, 3))
    ga = np.zeros_like(gc) if with_abs else None
    sa = np.zeros((P, K, 5)) if with_abs else None
    L.orc_blend_bwd(P, K, _p(p2f, _i64p), _p(zb, _f64p), _p(ba, _f64p), _p(di, _f64p), _p(fa, _i64p),
                    _p(co, _f64p), sigma, gamma, znear, zfar, _p(bgv, _f64p), int(mode), eps,
                    _p(g, _f64p), _p(gz, _f64p), _p(gb, _f64p), _p(gd, _f64p), _p(gc, _f64p), _p(ga, _f64p),
                    _p(sa, _f64p))
    out = (gz.reshape(*lead, K), gb.reshape(*lead, K, 3), gd.reshape(*lead, K), gc)
    if not with_abs:
        return out
    return out + (ga, sa[..., 1].reshape(*lead, K), sa[..., 2:].reshape(*lead, K, 3), sa[..., 0].reshape(*lead, K))


def rast_bwd(m: Mesh, S, K, pix_to_face, grad_zbuf, grad_bary, grad_dists, blur=0.0, persp=True,
             clip=False, pixels=None, with_abs=False):
    """Adjoint of ``rasterize`` conditioned on ``pix_to_face``; returns grad_verts (V, 3)
    (and the per-component sums of |contribution| when ``with_abs``)."""
    L = _load()
    px, P = _pixels(pixels)
    if px is None:
        P = m.N * S * S
    p2f = _i(pix_to_face).reshape(P, K)
    gz = None if grad_zbuf is None else _d(grad_zbuf).reshape(P, K)
    gb = None if grad_bary is None else _d(grad_bary).reshape(P, K, 3)
    gd = None if grad_dists is None else _d(grad_dists).reshape(P, K)
    gv = np.zeros_like(m.verts)
    ga = np.zeros_like(gv) if with_abs else None
    L.orc_rast_bwd(*m._head(), m.N, _p(m.cams, _f64p), S, K, float(blur), int(persp), int(clip),
                   _p(px, _i64p), P, _p(p2f, _i64p), _p(gz, _f64p), _p(gb, _f64p), _p(gd, _f64p),
                   _p(gv, _f64p), _p(ga, _f64p))
    return (gv, ga) if with_abs else gv
