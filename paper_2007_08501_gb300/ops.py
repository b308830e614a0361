"""Thin ctypes binding of ``libmeshrast.so`` (C ABI: ``include/meshrast.h``).

Argument marshalling only: every function takes torch CUDA tensors (used as
device memory), checks dtype/device/contiguity, and passes raw pointers and
the current CUDA stream to the entry point of the same name.  All arithmetic
happens in the library's kernels.  There is no CPU fallback: a missing or
unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MESHRAST_OK = 0
MESHRAST_ERR_INVALID_ARG = -1
MESHRAST_ERR_WORKSPACE = -2
MESHRAST_ERR_UNSUPPORTED = -3
MESHRAST_ERR_CUDA = -4
MESHRAST_ERR_STATIC_TOO_LARGE = -5
STATIC_WORKSPACE_BYTES = 16 << 20

ST_BIN_OVERFLOW = 1
ST_BAD_INDEX = 2
ST_BAD_MESH_RANGE = 4
ST_NONFINITE = 8

BLEND_SIL = 0
BLEND_RGB = 1

EXPORTED = ("rast_workspace_bytes", "rast_mesh_fwd", "rast_mesh_bwd", "blend_fwd", "blend_bwd",
            "rast_query_status", "rast_bin_occupancy", "rast_strerror", "rast_mesh_fwd_static",
            "rast_query_static_status", "rast_workspace_bin_layout", "meshrast_fma_probe",
            "blend_rast_bwd", "rast_blend_fwd",
            "pts_workspace_bytes", "pts_rasterize_fwd", "pts_rasterize_bwd", "pts_composite_fwd",
            "pts_composite_bwd", "pts_bin_occupancy", "shade_fwd", "shade_bwd",
            "knn_workspace_bytes", "knn_points", "knn_points_bwd", "chamfer_fwd", "chamfer_bwd")

SHADE_FLAT, SHADE_GOURAUD, SHADE_PHONG = 0, 1, 2
SHADE_SOFTMAX, SHADE_HARD = 0, 1

PTS_ALPHA = 0
PTS_NORM = 1


class rast_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("image_size", ctypes.c_int32), ("faces_per_pixel", ctypes.c_int32),
                ("bin_size", ctypes.c_int32), ("max_faces_per_bin", ctypes.c_int32),
                ("perspective_correct", ctypes.c_int32), ("clip_barycentric_coords", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("blur_radius", ctypes.c_float), ("reserved_f", ctypes.c_float),
                ("max_bin_entries", ctypes.c_int64)]


class blend_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_float), ("gamma", ctypes.c_float), ("znear", ctypes.c_float),
                ("zfar", ctypes.c_float), ("bg", ctypes.c_float * 3), ("eps", ctypes.c_float),
                ("mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rast_bin_layout(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_int64), ("eff", ctypes.c_int64), ("offsets", ctypes.c_int64),
                ("lists", ctypes.c_int64), ("nb", ctypes.c_int64), ("NB", ctypes.c_int64),
                ("capacity", ctypes.c_int64), ("bytes", ctypes.c_int64), ("redo", ctypes.c_int64),
                ("order", ctypes.c_int64)]


class MeshRastError(RuntimeError):
    pass


_lib = None


class shade_params(ctypes.Structure):
    _fields_ = [("light", ctypes.c_float * 3), ("ambient", ctypes.c_float * 3), ("diffuse", ctypes.c_float * 3),
                ("specular", ctypes.c_float * 3), ("shininess", ctypes.c_float), ("shading", ctypes.c_int32),
                ("blend", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pts_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("image_size", ctypes.c_int32), ("points_per_pixel", ctypes.c_int32),
                ("bin_size", ctypes.c_int32), ("max_points_per_bin", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("radius", ctypes.c_float), ("reserved_f", ctypes.c_float), ("max_bin_entries", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Open the library (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise MeshRastError("libmeshrast.so is not built (run __graft_entry__.build()); "
                                "there is no fallback implementation")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER(rast_params)
    B = ctypes.POINTER(blend_params)
    L.rast_workspace_bytes.argtypes = [P, i64, i64]
    L.rast_workspace_bytes.restype = sz
    L.rast_mesh_fwd.argtypes = [P, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.rast_mesh_fwd.restype = ctypes.c_int
    L.rast_mesh_bwd.argtypes = [P, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.rast_mesh_bwd.restype = ctypes.c_int
    L.blend_fwd.argtypes = [B, i64, i64, i64, vp, vp, vp, vp, vp, i64, vp, i64, vp, vp]
    L.blend_fwd.restype = ctypes.c_int
    L.blend_bwd.argtypes = [B, i64, i64, i64, vp, vp, vp, vp, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp]
    L.blend_bwd.restype = ctypes.c_int
    L.rast_blend_fwd.argtypes = [P, B, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.rast_blend_fwd.restype = ctypes.c_int
    L.blend_rast_bwd.argtypes = [P, B, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.blend_rast_bwd.restype = ctypes.c_int
    L.rast_query_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), vp]
    L.rast_query_status.restype = ctypes.c_int
    L.rast_bin_occupancy.argtypes = [P, i64, i64, vp, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int64), vp]
    L.rast_bin_occupancy.restype = ctypes.c_int
    L.rast_mesh_fwd_static.argtypes = [P, vp, i64, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rast_mesh_fwd_static.restype = ctypes.c_int
    L.rast_query_static_status.argtypes = [ctypes.POINTER(ctypes.c_uint32), vp]
    L.rast_query_static_status.restype = ctypes.c_int
    L.rast_workspace_bin_layout.argtypes = [P, i64, i64, ctypes.POINTER(rast_bin_layout)]
    L.rast_workspace_bin_layout.restype = ctypes.c_int
    L.meshrast_fma_probe.argtypes = [vp, i64, ctypes.c_int32, vp]
    L.meshrast_fma_probe.restype = ctypes.c_int
    H = ctypes.POINTER(shade_params)
    L.shade_fwd.argtypes = [B, H, i64, i64, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp]
    L.shade_fwd.restype = ctypes.c_int
    L.shade_bwd.argtypes = [B, H, i64, i64, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp,
                            vp, vp]
    L.shade_bwd.restype = ctypes.c_int
    Q = ctypes.POINTER(pts_params)
    L.pts_workspace_bytes.argtypes = [Q, i64]
    L.pts_workspace_bytes.restype = sz
    L.pts_rasterize_fwd.argtypes = [Q, vp, i64, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.pts_rasterize_fwd.restype = ctypes.c_int
    L.pts_rasterize_bwd.argtypes = [Q, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.pts_rasterize_bwd.restype = ctypes.c_int
    L.pts_composite_fwd.argtypes = [Q, ctypes.c_int32, vp, vp, vp, i64, ctypes.c_int32, vp, vp]
    L.pts_composite_fwd.restype = ctypes.c_int
    L.pts_composite_bwd.argtypes = [Q, ctypes.c_int32, vp, vp, vp, i64, ctypes.c_int32, vp, vp, vp, vp]
    L.pts_composite_bwd.restype = ctypes.c_int
    L.pts_bin_occupancy.argtypes = [Q, i64, vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), vp]
    L.pts_bin_occupancy.restype = ctypes.c_int
    L.rast_strerror.argtypes = [ctypes.c_int]
    L.rast_strerror.restype = ctypes.c_char_p
    i32 = ctypes.c_int32
    L.knn_workspace_bytes.argtypes = [i64]
    L.knn_workspace_bytes.restype = sz
    L.knn_points.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, i64, i32, i32, vp, vp, vp, sz, vp]
    L.knn_points.restype = ctypes.c_int
    L.knn_points_bwd.argtypes = [vp, i64, vp, i64, i32, i32, vp, vp, vp, vp, vp]
    L.knn_points_bwd.restype = ctypes.c_int
    L.chamfer_fwd.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.chamfer_fwd.restype = ctypes.c_int
    L.chamfer_bwd.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp]
    L.chamfer_bwd.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != MESHRAST_OK:
        msg = load().rast_strerror(rc).decode()
        raise MeshRastError("%s failed: %s (%d)" % (what, msg, rc))


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise MeshRastError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise MeshRastError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise MeshRastError("%s must be contiguous" % name)
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


# The C ABI trusts the sizes it derives from the parameters and the leading
# dimensions; a tensor too small for them is refused here instead of being
# written past its end.
def _atleast(t, n, name):
    if t is not None and t.numel() < n:
        raise MeshRastError("%s holds %d elements, the call needs %d" % (name, t.numel(), n))


def _n(t):
    return t.numel() if t is not None else 0


def _rows_of(t, width, name):
    if t is not None and (t.dim() != 2 or t.shape[1] != width):
        raise MeshRastError("%s must be (rows, %d), got %s" % (name, width, tuple(t.shape)))


def _batch_inputs(N, verts, faces, first, count, cams, vname="verts"):
    _rows_of(verts, 3, vname)
    _rows_of(faces, 3, "faces")
    _atleast(first, N, "first index per image")
    _atleast(count, N, "count per image")
    _atleast(cams, 16 * N, "cams")


def _slots(N, S, K, names_and_tensors):
    slots = int(N) * int(S) * int(S) * int(K)
    for name, t in names_and_tensors:
        _atleast(t, 3 * slots if "bary" in name else slots, name)


def _image(t, N, S, C, name):
    _atleast(t, int(N) * int(S) * int(S) * int(C), name)


def make_rast_params(N, image_size, K, blur_radius=0.0, bin_size=16, max_faces_per_bin=1024,
                     perspective_correct=True, clip_barycentric_coords=False, max_bin_entries=0):
    p = rast_params()
    p.N, p.image_size, p.faces_per_pixel = int(N), int(image_size), int(K)
    p.bin_size, p.max_faces_per_bin = int(bin_size), int(max_faces_per_bin)
    p.perspective_correct = int(bool(perspective_correct))
    p.clip_barycentric_coords = int(bool(clip_barycentric_coords))
    p.reserved = 0
    p.blur_radius = float(blur_radius)
    p.reserved_f = 0.0
    p.max_bin_entries = int(max_bin_entries)
    return p


def make_blend_params(sigma=1e-4, gamma=1e-4, znear=0.1, zfar=100.0, bg=(1.0, 1.0, 1.0), eps=1e-10,
                      mode=BLEND_RGB):
    b = blend_params()
    b.sigma, b.gamma, b.znear, b.zfar = float(sigma), float(gamma), float(znear), float(zfar)
    b.bg[0], b.bg[1], b.bg[2] = (float(x) for x in bg)
    b.eps = float(eps)
    b.mode = int(mode)
    b.reserved = 0
    return b


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def rast_workspace_bytes(p: rast_params, V: int, F: int) -> int:
    n = load().rast_workspace_bytes(ctypes.byref(p), int(V), int(F))
    if n == 0:
        raise MeshRastError("rast_workspace_bytes: invalid or unsupported parameters")
    return int(n)


def rast_mesh_fwd(p, verts, faces, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists, workspace,
                  stream=None):
    _batch_inputs(p.N, verts, faces, first_face, num_faces, cams)
    _slots(p.N, p.image_size, p.faces_per_pixel,
           (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    rc = load().rast_mesh_fwd(
        ctypes.byref(p), _ptr(verts, torch.float32, "verts"), verts.shape[0],
        _ptr(faces, torch.int64, "faces"), faces.shape[0],
        _ptr(first_face, torch.int64, "first_face"), _ptr(num_faces, torch.int64, "num_faces"),
        _ptr(cams, torch.float32, "cams"),
        _ptr(pix_to_face, torch.int64, "pix_to_face"), _ptr(zbuf, torch.float32, "zbuf"),
        _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"),
        _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "rast_mesh_fwd")


def rast_mesh_fwd_static(p, verts, faces, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists,
                         stream=None, check=True):
    """rast_mesh_fwd without a workspace argument, for callers that cannot allocate
    device memory: the library uses its own built-in 16 MiB device array.  Returns
    the C return code (raises on error when ``check``)."""
    _batch_inputs(p.N, verts, faces, first_face, num_faces, cams)
    _slots(p.N, p.image_size, p.faces_per_pixel,
           (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    rc = load().rast_mesh_fwd_static(
        ctypes.byref(p), _ptr(verts, torch.float32, "verts"), verts.shape[0],
        _ptr(faces, torch.int64, "faces"), faces.shape[0],
        _ptr(first_face, torch.int64, "first_face"), _ptr(num_faces, torch.int64, "num_faces"),
        _ptr(cams, torch.float32, "cams"),
        _ptr(pix_to_face, torch.int64, "pix_to_face"), _ptr(zbuf, torch.float32, "zbuf"),
        _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"), _stream(stream))
    if check:
        _check(rc, "rast_mesh_fwd_static")
    return rc


def rast_query_static_status(stream=None) -> int:
    """Status bits left by the last rast_mesh_fwd_static call on this device (syncs the stream)."""
    v = ctypes.c_uint32(0)
    _check(load().rast_query_static_status(ctypes.byref(v), _stream(stream)), "rast_query_static_status")
    return int(v.value)


def fma_probe(out, blocks, iters, stream=None):
    """Enqueue the FP32 FMA throughput probe; returns the FLOPs it performs."""
    _atleast(out, blocks * 256, "out")
    _check(load().meshrast_fma_probe(_ptr(out, torch.float32, "out"), int(blocks), int(iters), _stream(stream)),
           "meshrast_fma_probe")
    return blocks * 256 * 8 * 16 * iters * 2


def rast_workspace_bin_layout(p, V, F) -> dict:
    """Byte offsets of the bin counts, clamped counts, offsets and lists in the workspace
    (binned parameters), with nb, NB, capacity and the workspace size."""
    out = rast_bin_layout()
    _check(load().rast_workspace_bin_layout(ctypes.byref(p), int(V), int(F), ctypes.byref(out)),
           "rast_workspace_bin_layout")
    return {k: int(getattr(out, k)) for k, _ in rast_bin_layout._fields_}


def rast_mesh_bwd(p, verts, faces, first_face, num_faces, cams, pix_to_face, grad_zbuf, grad_bary, grad_dists,
                  grad_verts, workspace, stream=None):
    _batch_inputs(p.N, verts, faces, first_face, num_faces, cams)
    _slots(p.N, p.image_size, p.faces_per_pixel, (("pix_to_face", pix_to_face), ("grad_zbuf", grad_zbuf),
                                                  ("grad_bary", grad_bary), ("grad_dists", grad_dists)))
    _atleast(grad_verts, _n(verts), "grad_verts")
    rc = load().rast_mesh_bwd(
        ctypes.byref(p), _ptr(verts, torch.float32, "verts"), verts.shape[0],
        _ptr(faces, torch.int64, "faces"), faces.shape[0],
        _ptr(first_face, torch.int64, "first_face"), _ptr(num_faces, torch.int64, "num_faces"),
        _ptr(cams, torch.float32, "cams"), _ptr(pix_to_face, torch.int64, "pix_to_face"),
        _ptr(grad_zbuf, torch.float32, "grad_zbuf"), _ptr(grad_bary, torch.float32, "grad_bary"),
        _ptr(grad_dists, torch.float32, "grad_dists"), _ptr(grad_verts, torch.float32, "grad_verts"),
        _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "rast_mesh_bwd")


def blend_fwd(bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, vert_colors, image, stream=None):
    _slots(N, S, K, (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    _rows_of(faces, 3, "faces")
    _rows_of(vert_colors, 3, "vert_colors")
    _image(image, N, S, 4, "image")
    F = faces.shape[0] if faces is not None else 0
    V = vert_colors.shape[0] if vert_colors is not None else 0
    rc = load().blend_fwd(ctypes.byref(bp), int(N), int(S), int(K), _ptr(pix_to_face, torch.int64, "pix_to_face"),
                          _ptr(zbuf, torch.float32, "zbuf"), _ptr(bary, torch.float32, "bary"),
                          _ptr(dists, torch.float32, "dists"), _ptr(faces, torch.int64, "faces"), F,
                          _ptr(vert_colors, torch.float32, "vert_colors"), V, _ptr(image, torch.float32, "image"),
                          _stream(stream))
    _check(rc, "blend_fwd")


def blend_bwd(bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, vert_colors, grad_image, grad_zbuf, grad_bary,
              grad_dists, grad_vert_colors, stream=None):
    _slots(N, S, K, (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists),
                     ("grad_zbuf", grad_zbuf), ("grad_bary", grad_bary), ("grad_dists", grad_dists)))
    _rows_of(faces, 3, "faces")
    _rows_of(vert_colors, 3, "vert_colors")
    _image(grad_image, N, S, 4, "grad_image")
    if vert_colors is not None:
        _atleast(grad_vert_colors, vert_colors.numel(), "grad_vert_colors")
    F = faces.shape[0] if faces is not None else 0
    V = vert_colors.shape[0] if vert_colors is not None else 0
    rc = load().blend_bwd(ctypes.byref(bp), int(N), int(S), int(K), _ptr(pix_to_face, torch.int64, "pix_to_face"),
                          _ptr(zbuf, torch.float32, "zbuf"), _ptr(bary, torch.float32, "bary"),
                          _ptr(dists, torch.float32, "dists"), _ptr(faces, torch.int64, "faces"), F,
                          _ptr(vert_colors, torch.float32, "vert_colors"), V,
                          _ptr(grad_image, torch.float32, "grad_image"), _ptr(grad_zbuf, torch.float32, "grad_zbuf"),
                          _ptr(grad_bary, torch.float32, "grad_bary"), _ptr(grad_dists, torch.float32, "grad_dists"),
                          _ptr(grad_vert_colors, torch.float32, "grad_vert_colors"), _stream(stream))
    _check(rc, "blend_bwd")


def rast_blend_fwd(p, bp, verts, faces, first_face, num_faces, cams, vert_colors, pix_to_face, zbuf, bary, dists,
                   image, workspace, stream=None):
    """rast_mesh_fwd and blend_fwd in one call (the fine pass blends as it writes)."""
    _batch_inputs(p.N, verts, faces, first_face, num_faces, cams)
    _slots(p.N, p.image_size, p.faces_per_pixel,
           (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    _atleast(vert_colors, _n(verts), "vert_colors")
    _image(image, p.N, p.image_size, 4, "image")
    rc = load().rast_blend_fwd(
        ctypes.byref(p), ctypes.byref(bp), _ptr(verts, torch.float32, "verts"), verts.shape[0],
        _ptr(faces, torch.int64, "faces"), faces.shape[0],
        _ptr(first_face, torch.int64, "first_face"), _ptr(num_faces, torch.int64, "num_faces"),
        _ptr(cams, torch.float32, "cams"), _ptr(vert_colors, torch.float32, "vert_colors"),
        _ptr(pix_to_face, torch.int64, "pix_to_face"), _ptr(zbuf, torch.float32, "zbuf"),
        _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"), _ptr(image, torch.float32, "image"),
        _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "rast_blend_fwd")


def blend_rast_bwd(p, bp, verts, faces, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists, vert_colors,
                   grad_image, grad_verts, grad_vert_colors, workspace, stream=None):
    """blend_bwd followed by rast_mesh_bwd in one pass (fragment gradients stay in registers)."""
    _batch_inputs(p.N, verts, faces, first_face, num_faces, cams)
    _slots(p.N, p.image_size, p.faces_per_pixel,
           (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    _atleast(vert_colors, _n(verts), "vert_colors")
    _image(grad_image, p.N, p.image_size, 4, "grad_image")
    _atleast(grad_verts, _n(verts), "grad_verts")
    _atleast(grad_vert_colors, _n(verts), "grad_vert_colors")
    rc = load().blend_rast_bwd(
        ctypes.byref(p), ctypes.byref(bp), _ptr(verts, torch.float32, "verts"), verts.shape[0],
        _ptr(faces, torch.int64, "faces"), faces.shape[0],
        _ptr(first_face, torch.int64, "first_face"), _ptr(num_faces, torch.int64, "num_faces"),
        _ptr(cams, torch.float32, "cams"), _ptr(pix_to_face, torch.int64, "pix_to_face"),
        _ptr(zbuf, torch.float32, "zbuf"), _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"),
        _ptr(vert_colors, torch.float32, "vert_colors"), _ptr(grad_image, torch.float32, "grad_image"),
        _ptr(grad_verts, torch.float32, "grad_verts"), _ptr(grad_vert_colors, torch.float32, "grad_vert_colors"),
        _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "blend_rast_bwd")


def rast_query_status(workspace, stream=None) -> int:
    v = ctypes.c_uint32(0)
    _check(load().rast_query_status(_ptr(workspace, None, "workspace"), ctypes.byref(v), _stream(stream)),
           "rast_query_status")
    return int(v.value)


def rast_bin_occupancy(p, V, F, workspace, stream=None):
    mc = ctypes.c_int32(0)
    tot = ctypes.c_int64(0)
    _check(load().rast_bin_occupancy(ctypes.byref(p), int(V), int(F), _ptr(workspace, None, "workspace"),
                                     ctypes.byref(mc), ctypes.byref(tot), _stream(stream)), "rast_bin_occupancy")
    return int(mc.value), int(tot.value)


def rast_strerror(code: int) -> str:
    return load().rast_strerror(int(code)).decode()


# ---------------------------------------------------------------------------
# allocation helpers (torch is the device-memory allocator)
# ---------------------------------------------------------------------------
def alloc_workspace(p, V, F, device="cuda"):
    n = rast_workspace_bytes(p, V, F)
    # uint8 storage from the caching allocator is 512-byte aligned
    ws = torch.empty(n, dtype=torch.uint8, device=device)
    assert ws.data_ptr() % 256 == 0
    return ws


def alloc_fragments(N, S, K, device="cuda"):
    return (torch.empty((N, S, S, K), dtype=torch.int64, device=device),
            torch.empty((N, S, S, K), dtype=torch.float32, device=device),
            torch.empty((N, S, S, K, 3), dtype=torch.float32, device=device),
            torch.empty((N, S, S, K), dtype=torch.float32, device=device))


# ---------------------------------------------------------------------------
# point clouds (include/points.h)
# ---------------------------------------------------------------------------
def make_pts_params(N, image_size, K, radius, bin_size=16, max_points_per_bin=4096, max_bin_entries=0):
    return pts_params(int(N), int(image_size), int(K), int(bin_size), int(max_points_per_bin), 0, float(radius), 0.0,
                      int(max_bin_entries))


def pts_workspace_bytes(p, P):
    return int(load().pts_workspace_bytes(ctypes.byref(p), int(P)))


def alloc_pts_workspace(p, P, device="cuda"):
    n = pts_workspace_bytes(p, P)
    if n == 0:
        raise MeshRastError("pts_workspace_bytes: invalid or unsupported parameters")
    return torch.empty(n, dtype=torch.uint8, device=device)


def alloc_pts_fragments(N, S, K, device="cuda"):
    return (torch.empty((N, S, S, K), dtype=torch.int64, device=device),
            torch.empty((N, S, S, K), dtype=torch.float32, device=device),
            torch.empty((N, S, S, K), dtype=torch.float32, device=device))


def pts_rasterize_fwd(p, points, first_point, num_points, cams, idx, zbuf, dists, workspace, stream=None):
    _batch_inputs(p.N, points, None, first_point, num_points, cams, "points")
    _slots(p.N, p.image_size, p.points_per_pixel, (("idx", idx), ("zbuf", zbuf), ("dists", dists)))
    rc = load().pts_rasterize_fwd(
        ctypes.byref(p), _ptr(points, torch.float32, "points"), points.shape[0],
        _ptr(first_point, torch.int64, "first_point"), _ptr(num_points, torch.int64, "num_points"),
        _ptr(cams, torch.float32, "cams"), _ptr(idx, torch.int64, "idx"), _ptr(zbuf, torch.float32, "zbuf"),
        _ptr(dists, torch.float32, "dists"), _ptr(workspace, None, "workspace"),
        workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "pts_rasterize_fwd")


def pts_rasterize_bwd(p, points, first_point, num_points, cams, idx, grad_zbuf, grad_dists, grad_points, workspace,
                      stream=None):
    _batch_inputs(p.N, points, None, first_point, num_points, cams, "points")
    _slots(p.N, p.image_size, p.points_per_pixel, (("idx", idx), ("grad_zbuf", grad_zbuf), ("grad_dists", grad_dists)))
    _atleast(grad_points, _n(points), "grad_points")
    rc = load().pts_rasterize_bwd(
        ctypes.byref(p), _ptr(points, torch.float32, "points"), points.shape[0],
        _ptr(first_point, torch.int64, "first_point"), _ptr(num_points, torch.int64, "num_points"),
        _ptr(cams, torch.float32, "cams"), _ptr(idx, torch.int64, "idx"), _ptr(grad_zbuf, torch.float32, "grad_zbuf"),
        _ptr(grad_dists, torch.float32, "grad_dists"), _ptr(grad_points, torch.float32, "grad_points"),
        _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "pts_rasterize_bwd")


def pts_composite_fwd(p, mode, idx, dists, features, image, stream=None):
    _slots(p.N, p.image_size, p.points_per_pixel, (("idx", idx), ("dists", dists)))
    if features.dim() != 2:
        raise MeshRastError("features must be (P, D)")
    _image(image, p.N, p.image_size, features.shape[1], "image")
    rc = load().pts_composite_fwd(ctypes.byref(p), int(mode), _ptr(idx, torch.int64, "idx"),
                                  _ptr(dists, torch.float32, "dists"), _ptr(features, torch.float32, "features"),
                                  features.shape[0], features.shape[1], _ptr(image, torch.float32, "image"),
                                  _stream(stream))
    _check(rc, "pts_composite_fwd")


def pts_composite_bwd(p, mode, idx, dists, features, grad_image, grad_dists, grad_features, stream=None):
    _slots(p.N, p.image_size, p.points_per_pixel, (("idx", idx), ("dists", dists), ("grad_dists", grad_dists)))
    if features.dim() != 2:
        raise MeshRastError("features must be (P, D)")
    _image(grad_image, p.N, p.image_size, features.shape[1], "grad_image")
    _atleast(grad_features, features.numel(), "grad_features")
    rc = load().pts_composite_bwd(ctypes.byref(p), int(mode), _ptr(idx, torch.int64, "idx"),
                                  _ptr(dists, torch.float32, "dists"), _ptr(features, torch.float32, "features"),
                                  features.shape[0], features.shape[1], _ptr(grad_image, torch.float32, "grad_image"),
                                  _ptr(grad_dists, torch.float32, "grad_dists"),
                                  _ptr(grad_features, torch.float32, "grad_features"), _stream(stream))
    _check(rc, "pts_composite_bwd")


def pts_bin_occupancy(p, P, workspace, stream=None):
    mc = ctypes.c_int32(0)
    tot = ctypes.c_int64(0)
    _check(load().pts_bin_occupancy(ctypes.byref(p), int(P), _ptr(workspace, None, "workspace"), ctypes.byref(mc),
                                    ctypes.byref(tot), _stream(stream)), "pts_bin_occupancy")
    return int(mc.value), int(tot.value)


# ---------------------------------------------------------------------------
# lit shading (flat / Gouraud / Phong, softmax or hard blend)
# ---------------------------------------------------------------------------
def make_shade_params(light, ambient=(0.5, 0.5, 0.5), diffuse=(0.3, 0.3, 0.3), specular=(0.2, 0.2, 0.2),
                      shininess=64.0, shading=SHADE_PHONG, blend=SHADE_SOFTMAX):
    f3 = lambda v: (ctypes.c_float * 3)(*[float(x) for x in v])
    return shade_params(f3(light), f3(ambient), f3(diffuse), f3(specular), float(shininess), int(shading), int(blend),
                        0)


def shade_fwd(bp, sp, N, S, K, pix_to_face, zbuf, bary, dists, faces, verts, normals, vert_colors, cams, image,
              stream=None):
    _slots(N, S, K, (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists)))
    _rows_of(faces, 3, "faces")
    _rows_of(verts, 3, "verts")
    _atleast(normals, _n(verts), "normals")
    _atleast(vert_colors, _n(verts), "vert_colors")
    _atleast(cams, 16 * int(N), "cams")
    _image(image, N, S, 4, "image")
    rc = load().shade_fwd(ctypes.byref(bp), ctypes.byref(sp), int(N), int(S), int(K),
                          _ptr(pix_to_face, torch.int64, "pix_to_face"), _ptr(zbuf, torch.float32, "zbuf"),
                          _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"),
                          _ptr(faces, torch.int64, "faces"), faces.shape[0], _ptr(verts, torch.float32, "verts"),
                          _ptr(normals, torch.float32, "normals"), _ptr(vert_colors, torch.float32, "vert_colors"),
                          verts.shape[0], _ptr(cams, torch.float32, "cams"), _ptr(image, torch.float32, "image"),
                          _stream(stream))
    _check(rc, "shade_fwd")


def shade_bwd(bp, sp, N, S, K, pix_to_face, zbuf, bary, dists, faces, verts, normals, vert_colors, cams, grad_image,
              grad_zbuf, grad_bary, grad_dists, grad_verts, grad_normals, grad_vert_colors, stream=None):
    _slots(N, S, K, (("pix_to_face", pix_to_face), ("zbuf", zbuf), ("bary", bary), ("dists", dists),
                     ("grad_zbuf", grad_zbuf), ("grad_bary", grad_bary), ("grad_dists", grad_dists)))
    _rows_of(faces, 3, "faces")
    _rows_of(verts, 3, "verts")
    for t, name in ((normals, "normals"), (vert_colors, "vert_colors"), (grad_verts, "grad_verts"),
                    (grad_normals, "grad_normals"), (grad_vert_colors, "grad_vert_colors")):
        _atleast(t, _n(verts), name)
    _atleast(cams, 16 * int(N), "cams")
    _image(grad_image, N, S, 4, "grad_image")
    rc = load().shade_bwd(ctypes.byref(bp), ctypes.byref(sp), int(N), int(S), int(K),
                          _ptr(pix_to_face, torch.int64, "pix_to_face"), _ptr(zbuf, torch.float32, "zbuf"),
                          _ptr(bary, torch.float32, "bary"), _ptr(dists, torch.float32, "dists"),
                          _ptr(faces, torch.int64, "faces"), faces.shape[0], _ptr(verts, torch.float32, "verts"),
                          _ptr(normals, torch.float32, "normals"), _ptr(vert_colors, torch.float32, "vert_colors"),
                          verts.shape[0], _ptr(cams, torch.float32, "cams"),
                          _ptr(grad_image, torch.float32, "grad_image"), _ptr(grad_zbuf, torch.float32, "grad_zbuf"),
                          _ptr(grad_bary, torch.float32, "grad_bary"), _ptr(grad_dists, torch.float32, "grad_dists"),
                          _ptr(grad_verts, torch.float32, "grad_verts"),
                          _ptr(grad_normals, torch.float32, "grad_normals"),
                          _ptr(grad_vert_colors, torch.float32, "grad_vert_colors"), _stream(stream))
    _check(rc, "shade_bwd")


# ---------------------------------------------------------------------------
# exact K nearest neighbours and the Chamfer loss (packed point-cloud batches)
# ---------------------------------------------------------------------------
def knn_workspace_bytes(N):
    return int(load().knn_workspace_bytes(int(N)))


def alloc_knn_workspace(N, device="cuda"):
    """256-byte aligned device workspace for knn_points / chamfer_fwd over N clouds."""
    n = max(knn_workspace_bytes(N), 256)
    return torch.empty(n // 8, dtype=torch.int64, device=device)


def _ws(workspace):
    return _ptr(workspace, None, "workspace"), workspace.numel() * workspace.element_size()


def _need(t, n, name):
    """The C ABI trusts the sizes it derives from the shapes: a tensor with
    another element count is refused here (a NULL pointer is left to the call)."""
    if t is not None and t.numel() != n:
        raise MeshRastError("%s must hold %d elements, got %d" % (name, n, t.numel()))


def _clouds(p, first, length, name):
    if p.dim() != 2:
        raise MeshRastError("%s must be (points, D)" % name)
    _need(length, first.numel(), "the cloud lengths of " + name)


def knn_points(p1, first1, len1, p2, first2, len2, K, idx, dists, workspace, stream=None):
    """idx (P1, K) int64 and dists (P1, K) float32 are written (global rows of p2)."""
    D = p1.shape[1]
    if p2.shape[1] != D:
        raise MeshRastError("p1 and p2 must have the same dimension")
    _clouds(p1, first1, len1, "p1")
    _clouds(p2, first2, len2, "p2")
    _need(first2, first1.numel(), "first2")
    _need(idx, p1.shape[0] * int(K), "idx")
    _need(dists, p1.shape[0] * int(K), "dists")
    w, wb = _ws(workspace)
    rc = load().knn_points(_ptr(p1, torch.float32, "p1"), p1.shape[0], _ptr(first1, torch.int64, "first1"),
                           _ptr(len1, torch.int64, "len1"), _ptr(p2, torch.float32, "p2"), p2.shape[0],
                           _ptr(first2, torch.int64, "first2"), _ptr(len2, torch.int64, "len2"), first1.shape[0], D,
                           int(K), _ptr(idx, torch.int64, "idx"), _ptr(dists, torch.float32, "dists"), w, wb,
                           _stream(stream))
    _check(rc, "knn_points")


def knn_points_bwd(p1, p2, idx, grad_dists, grad_p1, grad_p2, stream=None):
    if idx.dim() != 2 or idx.shape[0] != p1.shape[0]:
        raise MeshRastError("idx must be (P1, K)")
    _need(grad_dists, idx.numel(), "grad_dists")
    _need(grad_p1, p1.numel(), "grad_p1")
    _need(grad_p2, p2.numel(), "grad_p2")
    rc = load().knn_points_bwd(_ptr(p1, torch.float32, "p1"), p1.shape[0], _ptr(p2, torch.float32, "p2"), p2.shape[0],
                               p1.shape[1], idx.shape[1], _ptr(idx, torch.int64, "idx"),
                               _ptr(grad_dists, torch.float32, "grad_dists"), _ptr(grad_p1, torch.float32, "grad_p1"),
                               _ptr(grad_p2, torch.float32, "grad_p2"), _stream(stream))
    _check(rc, "knn_points_bwd")


def chamfer_fwd(p, first1, len1, q, first2, len2, idx_pq, d_pq, idx_qp, d_qp, loss_per_pair, loss, workspace,
                stream=None):
    D = p.shape[1]
    if q.shape[1] != D:
        raise MeshRastError("p and q must have the same dimension")
    _clouds(p, first1, len1, "p")
    _clouds(q, first2, len2, "q")
    _need(first2, first1.numel(), "first2")
    for t, n, name in ((idx_pq, p.shape[0], "idx_pq"), (d_pq, p.shape[0], "d_pq"), (idx_qp, q.shape[0], "idx_qp"),
                       (d_qp, q.shape[0], "d_qp"), (loss_per_pair, first1.numel(), "loss_per_pair"), (loss, 1, "loss")):
        _need(t, n, name)
    w, wb = _ws(workspace)
    rc = load().chamfer_fwd(_ptr(p, torch.float32, "p"), p.shape[0], _ptr(first1, torch.int64, "first1"),
                            _ptr(len1, torch.int64, "len1"), _ptr(q, torch.float32, "q"), q.shape[0],
                            _ptr(first2, torch.int64, "first2"), _ptr(len2, torch.int64, "len2"), first1.shape[0], D,
                            _ptr(idx_pq, torch.int64, "idx_pq"), _ptr(d_pq, torch.float32, "d_pq"),
                            _ptr(idx_qp, torch.int64, "idx_qp"), _ptr(d_qp, torch.float32, "d_qp"),
                            _ptr(loss_per_pair, torch.float32, "loss_per_pair"), _ptr(loss, torch.float32, "loss"),
                            w, wb, _stream(stream))
    _check(rc, "chamfer_fwd")


def chamfer_bwd(p, first1, len1, q, first2, len2, idx_pq, idx_qp, grad_loss, grad_per_pair, grad_p, grad_q,
                stream=None):
    _clouds(p, first1, len1, "p")
    _clouds(q, first2, len2, "q")
    _need(first2, first1.numel(), "first2")
    for t, n, name in ((idx_pq, p.shape[0], "idx_pq"), (idx_qp, q.shape[0], "idx_qp"), (grad_loss, 1, "grad_loss"),
                       (grad_per_pair, first1.numel(), "grad_per_pair"), (grad_p, p.numel(), "grad_p"),
                       (grad_q, q.numel(), "grad_q")):
        _need(t, n, name)
    rc = load().chamfer_bwd(_ptr(p, torch.float32, "p"), p.shape[0], _ptr(first1, torch.int64, "first1"),
                            _ptr(len1, torch.int64, "len1"), _ptr(q, torch.float32, "q"), q.shape[0],
                            _ptr(first2, torch.int64, "first2"), _ptr(len2, torch.int64, "len2"), first1.shape[0],
                            p.shape[1], _ptr(idx_pq, torch.int64, "idx_pq"), _ptr(idx_qp, torch.int64, "idx_qp"),
                            _ptr(grad_loss, torch.float32, "grad_loss"),
                            _ptr(grad_per_pair, torch.float32, "grad_per_pair"), _ptr(grad_p, torch.float32, "grad_p"),
                            _ptr(grad_q, torch.float32, "grad_q"), _stream(stream))
    _check(rc, "chamfer_bwd")
