"""CPU oracle for the Stage-II differentiable UV-PBR renderer (Sec. 5 of the paper).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package: it is
loaded by the test suite, by the smoke check and by the CPU-baseline leg of the
benchmark.  It shares no code with the CUDA library.

Two layers:

* ``decide.c`` (built into ``liboracle.so``): the discrete decisions, brute force, in the
  FP32 specification both sides implement (fixed-point raster, integer environment CDF,
  Philox4x32-10 sample streams, watertight ray/triangle tests against every triangle).
* ``shade.py``: the estimator of Eqs. 10-20 evaluated in FP64 with plain PyTorch CPU
  operations; gradients are torch.autograd's reverse-mode derivative of that definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

GUARDBAND = -4


def build(force: bool = False) -> str:
    """Compile decide.c into liboracle.so (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "decide.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", src, "-o", _LIB_PATH + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, u64 = ctypes.c_int, ctypes.c_uint64
        L.orc_philox.argtypes = [P, P, P]
        L.orc_sincos2pi_many.argtypes = [P, i32, P, P]
        L.orc_snap.argtypes = [P, i32, P, P, P]
        L.orc_snap.restype = i32
        L.orc_raster_pixels.argtypes = [P, i32, P, i32, P, i32, i32, i32, P, i32, P]
        L.orc_raster_pixels.restype = i32
        L.orc_raster_full.argtypes = [P, i32, P, i32, P, i32, i32, i32, P]
        L.orc_raster_full.restype = i32
        L.orc_coverage_counts.argtypes = [P, i32, P, i32, P, i32, i32, P, P]
        L.orc_coverage_counts.restype = i32
        L.orc_env_table.argtypes = [P, i32, i32, P, P]
        L.orc_env_table.restype = u64
        L.orc_light_dirs.argtypes = [P, P, i32, i32, i32, P]
        L.orc_trace.argtypes = [P, P, i32, P, P, i32, i32, P, P, P]
        L.orc_decide.argtypes = [P, P, i32, P, i32, i32, P, i32, i32, u64, i32, i32, i32, P, P, i32,
                                 P, P, P, P, P, P, P, P, P, P, P]
        L.orc_decide.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle buffers must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ thin wrappers

def philox(ctr, key):
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def sincos2pi(s):
    s = _c(s, np.float32).ravel()
    sn = np.zeros_like(s)
    cs = np.zeros_like(s)
    lib().orc_sincos2pi_many(_p(s), s.size, _p(sn), _p(cs))
    return sn, cs


def snap(V, cam):
    V = _c(V, np.float32)
    cam = _c(cam, np.float32)
    XY = np.zeros((V.shape[0], 2), np.int32)
    Zq = np.zeros(V.shape[0], np.uint32)
    st = lib().orc_snap(_p(V), V.shape[0], _p(cam), _p(XY), _p(Zq))
    return st, XY, Zq


def raster_full(V, F, cams, W, H):
    V, F, cams = _c(V, np.float32), _c(F, np.int32), _c(cams, np.float32)
    keys = np.zeros((cams.shape[0], H, W), np.uint64)
    st = lib().orc_raster_full(_p(V), V.shape[0], _p(F), F.shape[0], _p(cams), cams.shape[0], W, H, _p(keys))
    return st, keys


def raster_pixels(V, F, cams, W, H, pix):
    V, F, cams, pix = _c(V, np.float32), _c(F, np.int32), _c(cams, np.float32), _c(pix, np.int32)
    keys = np.zeros(pix.shape[0], np.uint64)
    st = lib().orc_raster_pixels(_p(V), V.shape[0], _p(F), F.shape[0], _p(cams), cams.shape[0], W, H,
                                 _p(pix), pix.shape[0], _p(keys))
    return st, keys


def coverage_counts(V, F, cam, W, H):
    V, F, cam = _c(V, np.float32), _c(F, np.int32), _c(cam, np.float32)
    front = np.zeros((H, W), np.int32)
    back = np.zeros((H, W), np.int32)
    st = lib().orc_coverage_counts(_p(V), V.shape[0], _p(F), F.shape[0], _p(cam), W, H, _p(front), _p(back))
    return st, front, back


class EnvTable:
    """Integer importance weights q [H*W], inclusive prefix cdf [H*W] and total Q."""

    def __init__(self, env):
        env = _c(env, np.float32)
        self.H, self.W = env.shape[:2]
        n = self.H * self.W
        self.q = np.zeros(n, np.uint32)
        self.cdf = np.zeros(n, np.uint64)
        self.Q = int(lib().orc_env_table(_p(env), self.W, self.H, _p(self.q), _p(self.cdf)))


def light_dirs(texels, xi, W, H):
    t = _c(texels, np.uint32).ravel()
    x = _c(xi, np.float32).reshape(-1, 2)
    out = np.zeros((t.size, 3), np.float32)
    lib().orc_light_dirs(_p(t), _p(x), t.size, W, H, _p(out))
    return out


def trace(V, F, O, D, closest: bool):
    V, F, O, D = _c(V, np.float32), _c(F, np.int32), _c(O, np.float32), _c(D, np.float32)
    n = O.shape[0]
    tri = np.zeros(n, np.int32)
    t = np.zeros(n, np.float32)
    front = np.zeros(n, np.int32)
    lib().orc_trace(_p(V), _p(F), F.shape[0], _p(O), _p(D), n, 1 if closest else 0, _p(tri), _p(t), _p(front))
    return (tri, t, front) if closest else tri.astype(bool)


class Decisions:
    """Per-pixel discrete decisions for a pixel list (see orc_decide in decide.c)."""

    def __init__(self, scene, table: EnvTable, pix, keys, V=None):
        V = _c(scene.V if V is None else V, np.float32)
        F = _c(scene.F, np.int32)
        cams = _c(scene.cams, np.float32)
        pix = _c(pix, np.int32)
        keys = _c(keys, np.uint64)
        P, Nd, Nb, Ns = pix.shape[0], scene.n_direct, max(scene.n_bounce, 0), max(scene.n_light, 0)
        self.pix, self.keys = pix, keys
        self.tri = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
        self.covered = self.tri != 0xFFFFFFFF
        self.dtex = np.zeros((P, Nd), np.int32)
        self.dxi = np.zeros((P, Nd, 2), np.float32)
        self.dvis = np.zeros((P, Nd), np.uint8)
        nb1, ns1 = max(Nb, 1), max(Ns, 1)
        self.stri = np.full((P, nb1), -1, np.int32)
        self.sb = np.zeros((P, nb1, 3), np.float64)
        self.sdir = np.zeros((P, nb1, 3), np.float32)
        self.sxi1 = np.zeros((P, nb1), np.float32)
        self.sgap = np.zeros((P, nb1), np.float32)
        self.ltex = np.full((P, nb1, ns1), -1, np.int32)
        self.lxi = np.zeros((P, nb1, ns1, 2), np.float32)
        self.lvis = np.zeros((P, nb1, ns1), np.uint8)
        lib().orc_decide(_p(V), _p(F), F.shape[0], _p(cams), scene.width, scene.height, _p(table.cdf),
                         table.W, table.H, int(scene.seed), Nd, Nb, Ns, _p(pix), _p(keys), P,
                         _p(self.dtex), _p(self.dxi), _p(self.dvis), _p(self.stri), _p(self.sb), _p(self.sdir),
                         _p(self.sxi1), _p(self.sgap), _p(self.ltex), _p(self.lxi), _p(self.lvis))
        if Nb == 0:
            self.stri = self.stri[:, :0]


def covered_pixels(keys):
    """(view, py, px) triples of every covered pixel of a [views, H, W] key image."""
    idx = np.argwhere((keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF))
    return idx.astype(np.int32)
