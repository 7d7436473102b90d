"""Plain CPU oracle of the path tracer with the shadow-receiving material (§III-D.2, §III-D.3, Eq. 7).

TEST INFRASTRUCTURE ONLY: only the tests may use this module; it shares no code with the CUDA library.
The arithmetic is in render_oracle.cpp (brute-force closest hits, FP32 without contraction)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import ipc

DIFFUSE, EMISSIVE, BACKGROUND, TRANSPARENT = 0, 1, 2, 3


def camera(eye, target, up, fov_deg, width, height):
    """Pinhole camera looking from eye at target: (13 floats: eye, fwd, right, up, tan(fov/2)), width, height."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    cam = np.concatenate([eye, f, r, u, [np.tan(np.radians(fov_deg) / 2)]]).astype(np.float32)
    return cam, int(width), int(height)


def render(x, tris, types, rgb, cam, spp=4, max_depth=2, n_shadow=8, lambda_s=0.8, eps=1e-5, seed=0):
    """Image (height, width, 3) float32 of the frame at vertex positions x."""
    lib = ipc.lib()
    f = lib.orc_render
    f.argtypes = [C.c_int, ipc.dp, C.c_int, ipc.ip, ipc.ip, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int,
                  C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_ulonglong, C.POINTER(C.c_float)]
    c, w, h = cam
    x = np.ascontiguousarray(x, np.float64)
    tris = np.ascontiguousarray(tris, np.int32)
    types = np.ascontiguousarray(types, np.int32)
    rgb = np.ascontiguousarray(rgb, np.float32)
    c = np.ascontiguousarray(c, np.float32)
    img = np.zeros((h, w, 3), np.float32)
    fp = C.POINTER(C.c_float)
    f(len(x), ipc._d(x), len(tris), ipc._i(tris), ipc._i(types), rgb.ctypes.data_as(fp), c.ctypes.data_as(fp), w, h,
      int(spp), int(max_depth), int(n_shadow), float(lambda_s), float(eps), int(seed), img.ctypes.data_as(fp))
    return img
