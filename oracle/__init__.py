"""FP64 CPU oracle for the Fireflies hot path (ctypes wrapper around ffo.c).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package.  The CUDA library never calls it and it never calls the CUDA
library; the two share no code.

Every function is pinned in ``tests/test_oracle_*.py`` against closed forms,
published values or facts printed in the paper (Sec. 2.2 Lorenz bifurcation
values, Hodgkin-Huxley resting gates, RK4 stability polynomial, ...).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffo.c")
_LIB = os.path.join(_HERE, "libffo.so")
_SRC32 = os.path.join(_HERE, "ffo_fp32.c")
_LIB32 = os.path.join(_HERE, "libffo32.so")

LINEAR, HARMONIC, WILSON_COWAN, LORENZ, HH3 = 0, 1, 2, 3, 4
RK4, EULER = 0, 1

_lib = None


def _compile(src, lib, deps, force):
    if force or not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(d) for d in deps):
        tmp = f"{lib}.{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)  # atomic: concurrent test workers never load a partial file
    return lib


def build(force: bool = False) -> str:
    """Compile ffo.c with gcc into oracle/libffo.so (no FMA contraction), and its
    single-precision evaluation ffo_fp32.c into oracle/libffo32.so."""
    _compile(_SRC32, _LIB32, [_SRC, _SRC32], force)
    return _compile(_SRC, _LIB, [_SRC], force)


def _load():
    global _lib
    if _lib is None:
        # FFO_LIB points the wrapper at another build of ffo.c (used by the mutation test,
        # which compiles deliberately broken copies into a temporary directory)
        path = os.environ.get("FFO_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.ffo_splitmix64.restype = ctypes.c_uint64
        lib.ffo_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.ffo_seed_group.restype = None
        lib.ffo_seed_group.argtypes = [ctypes.c_int, i64, i64, P, P, P, ctypes.c_uint64, P, i64]
        lib.ffo_linspace.restype = None
        lib.ffo_linspace.argtypes = [i64, i64, i64, P, ctypes.c_double, ctypes.c_double, P]
        lib.ffo_rhs.restype = ctypes.c_int
        lib.ffo_rhs.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P]
        lib.ffo_integrate.restype = ctypes.c_int
        lib.ffo_integrate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64, P, P,
                                      ctypes.c_int, ctypes.c_int, P, P, i64]
        lib.ffo_integrate_reset.restype = ctypes.c_int
        lib.ffo_integrate_reset.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, P, P, ctypes.c_int,
                                            ctypes.c_int, P, P, i64, i64, ctypes.c_int, P, P, ctypes.c_uint32,
                                            P, P, P, P, P, P, P]
        lib.ffo_jacobians.restype = ctypes.c_int
        lib.ffo_jacobians.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P]
        lib.ffo_tangent.restype = ctypes.c_int
        lib.ffo_tangent.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, P, P, ctypes.c_int, ctypes.c_int,
                                    P, P, i64, P, P, P]
        lib.ffo_count_escaped.restype = i64
        lib.ffo_count_escaped.argtypes = [ctypes.c_int, i64, i64, P, P]
        lib.ffo_splat2d.restype = None
        lib.ffo_splat2d.argtypes = [i64, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, P]
        lib.ffo_splat3d.restype = None
        lib.ffo_splat3d.argtypes = [i64, P, P, P, P, P, ctypes.c_int, ctypes.c_int, P]
        d, f, c_int = ctypes.c_double, ctypes.c_float, ctypes.c_int
        lib.ffo_sprites2d.restype = None
        lib.ffo_sprites2d.argtypes = [i64, P, P, P, P, d, d, d, d, c_int, c_int, f, d, P, P, P, P]
        lib.ffo_sprites3d.restype = None
        lib.ffo_sprites3d.argtypes = [i64, P, P, P, P, P, P, c_int, c_int, f, d, P, P, P, P]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def splitmix64(seed: int, n: int) -> int:
    """Output n (n >= 1) of the SplitMix64 stream seeded with ``seed``."""
    return int(_load().ffo_splitmix64(seed & (2**64 - 1), n & (2**64 - 1)))


def seed_group(dim, lo, hi, seed, count=None, j0=0, idx=None):
    """Initial conditions of group particles (float32, SoA [dim][count]).

    Particles ``j0 .. j0+count-1`` of the group, or the group-local indices
    ``idx`` if given.
    """
    lo = _c(lo, np.float64)
    hi = _c(hi, np.float64)
    if idx is not None:
        idx = _c(idx, np.int64)
        count = idx.size
    out = np.empty((dim, count), dtype=np.float32)
    _load().ffo_seed_group(dim, count, j0, _ptr(idx), _ptr(lo), _ptr(hi), seed & (2**64 - 1),
                           _ptr(out), count)
    return out


def linspace_param(P, lo, hi, i0=0, count=None, idx=None):
    """Per-particle parameter values (float32) for particles i0.. or idx of P."""
    if idx is not None:
        idx = _c(idx, np.int64)
        count = idx.size
    elif count is None:
        count = P - i0
    out = np.empty(count, dtype=np.float32)
    _load().ffo_linspace(P, i0, count, _ptr(idx), float(lo), float(hi), _ptr(out))
    return out


def rhs(rhs_id, x, params):
    """One evaluation of f(x, p) in FP64."""
    x = _c(x, np.float64)
    p = _c(params, np.float64)
    dx = np.empty_like(x)
    rc = _load().ffo_rhs(rhs_id, x.size, _ptr(x), _ptr(p), p.size, _ptr(dx))
    if rc != 0:
        raise ValueError("ffo_rhs: bad system id or size")
    return dx


def integrate(rhs_id, state, params, h, n_steps, method=RK4, pparam_index=-1, pparam=None):
    """Integrate SoA state [dim][P] (copied to float64) for n_steps; returns the new state.

    ``h`` is a scalar or a per-particle array of signed steps.
    """
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    if st.ndim == 1:
        st = st.reshape(-1, 1)
    dim, P = st.shape
    p = _c(params, np.float64)
    hh = np.broadcast_to(np.asarray(h, dtype=np.float64), (P,)).copy()
    pp = None if pparam is None else _c(pparam, np.float64)
    rc = _load().ffo_integrate(rhs_id, method, dim, P, P, _ptr(st), _ptr(p), p.size, pparam_index,
                               _ptr(pp), _ptr(hh), int(n_steps))
    if rc != 0:
        raise ValueError("ffo_integrate: bad arguments")
    return st


def integrate_parallel(rhs_id, state, params, h, n_steps, method=RK4, pparam_index=-1, pparam=None,
                       threads=None):
    """Same as :func:`integrate`, split over threads on disjoint particle ranges.

    The integrator itself stays the single-threaded C loop; ctypes releases the
    GIL during each call, so the ranges run concurrently.
    """
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    dim, P = st.shape
    threads = threads or os.cpu_count() or 1
    p = _c(params, np.float64)
    hh = np.broadcast_to(np.asarray(h, dtype=np.float64), (P,)).copy()
    pp = None if pparam is None else _c(pparam, np.float64)
    bounds = np.linspace(0, P, threads + 1).astype(np.int64)
    lib = _load()

    def work(t):
        a, b = int(bounds[t]), int(bounds[t + 1])
        if b <= a:
            return 0
        chunk = np.ascontiguousarray(st[:, a:b])
        ppc = None if pp is None else np.ascontiguousarray(pp[a:b])
        hc = np.ascontiguousarray(hh[a:b])
        rc = lib.ffo_integrate(rhs_id, method, dim, b - a, b - a, _ptr(chunk), _ptr(p), p.size,
                               pparam_index, _ptr(ppc), _ptr(hc), int(n_steps))
        st[:, a:b] = chunk
        return rc

    with ThreadPoolExecutor(max_workers=threads) as ex:
        rcs = list(ex.map(work, range(threads)))
    if any(rcs):
        raise ValueError("ffo_integrate: bad arguments")
    return st, threads


_lib32 = None


def integrate_fp32(rhs_id, state, params, h, n_steps, method=RK4, pparam_index=-1, pparam=None):
    """The oracle's integration evaluated in FP32 (ffo_fp32.c): state, parameters, steps and
    every intermediate in float32, elementary functions rounded once to float.  Not a parity
    reference -- a yardstick for the error any FP32 evaluation of the same formulas has
    against the FP64 oracle.  Returns the float32 state [dim][P]."""
    global _lib32
    if _lib32 is None:
        build()
        lib = ctypes.CDLL(_LIB32)
        P_, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.ffo_integrate.restype = ctypes.c_int
        lib.ffo_integrate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64, P_, P_, ctypes.c_int,
                                      ctypes.c_int, P_, P_, i64]
        _lib32 = lib
    st = np.array(state, dtype=np.float32, order="C", copy=True)
    if st.ndim == 1:
        st = st.reshape(-1, 1)
    dim, P = st.shape
    p = _c(params, np.float32)
    hh = np.broadcast_to(np.asarray(h, dtype=np.float32), (P,)).copy()
    pp = None if pparam is None else _c(pparam, np.float32)
    rc = _lib32.ffo_integrate(rhs_id, method, dim, P, P, _ptr(st), _ptr(p), p.size, pparam_index, _ptr(pp),
                              _ptr(hh), int(n_steps))
    if rc != 0:
        raise ValueError("ffo_integrate (fp32): bad arguments")
    return st


def integrate_reset(rhs_id, state, params, groups, dt, n_steps, step0=0, check_every=1, bounds=None,
                    max_age=0, age=None, resets=None, method=RK4, pparam_index=-1, pparam=None):
    """Integrate with the paper's particle reset (see ffo_integrate_reset).

    ``groups``: list of dicts with count, lo, hi, direction, seed (in particle order);
    ``bounds``: (lo[dim], hi[dim]) of the valid state box, or None.  Returns
    (state, age, resets); age/resets start from the given arrays (zeros by default).
    """
    st = np.array(state, dtype=np.float64, order="C", copy=True)
    dim, P = st.shape
    j = np.concatenate([np.arange(g["count"], dtype=np.int64) for g in groups])
    cnt = np.concatenate([np.full(g["count"], g["count"], np.int64) for g in groups])
    sd = np.concatenate([np.full(g["count"], g["seed"] & (2**64 - 1), np.uint64) for g in groups])
    lo = np.ascontiguousarray(np.concatenate([np.repeat(np.asarray(g["lo"], np.float64)[:, None], g["count"], 1)
                                              for g in groups], axis=1))
    hi = np.ascontiguousarray(np.concatenate([np.repeat(np.asarray(g["hi"], np.float64)[:, None], g["count"], 1)
                                              for g in groups], axis=1))
    h = np.concatenate([np.full(g["count"], g["direction"] * dt) for g in groups])
    age = np.zeros(P, np.uint32) if age is None else np.array(age, np.uint32)
    resets = np.zeros(P, np.uint32) if resets is None else np.array(resets, np.uint32)
    blo = bhi = None
    if bounds is not None:
        blo = np.asarray(bounds[0], np.float32)
        bhi = np.asarray(bounds[1], np.float32)
    p = _c(params, np.float64)
    pp = None if pparam is None else _c(pparam, np.float64)
    rc = _load().ffo_integrate_reset(rhs_id, method, dim, P, _ptr(st), _ptr(p), p.size, pparam_index, _ptr(pp),
                                     _ptr(h), int(n_steps), int(step0), int(check_every), _ptr(blo), _ptr(bhi),
                                     int(max_age), _ptr(j), _ptr(cnt), _ptr(sd), _ptr(lo), _ptr(hi), _ptr(age),
                                     _ptr(resets))
    if rc != 0:
        raise ValueError("ffo_integrate_reset: bad arguments")
    return st, age, resets


def jacobians(rhs_id, x, params):
    """(J, Fp): d f / d x (dim x dim) and d f / d p (dim x n_params) at x."""
    x = _c(x, np.float64)
    p = _c(params, np.float64)
    J = np.empty((x.size, x.size))
    Fp = np.empty((x.size, p.size))
    if _load().ffo_jacobians(rhs_id, x.size, _ptr(x), _ptr(p), p.size, _ptr(J), _ptr(Fp)) != 0:
        raise ValueError("ffo_jacobians: system without derivatives or bad size")
    return J, Fp


def tangent(rhs_id, x0, params, h, n_steps, pparam_index=-1, pparam=None, method=RK4):
    """Forward sensitivities: (x(T) [dim][P], S [P][dim][dim], Q [P][dim][n_params])."""
    x0 = _c(x0, np.float64)
    dim, P = x0.shape
    p = _c(params, np.float64)
    hh = np.broadcast_to(np.asarray(h, dtype=np.float64), (P,)).copy()
    pp = None if pparam is None else _c(pparam, np.float64)
    xT = np.empty_like(x0)
    S = np.empty((P, dim, dim))
    Q = np.empty((P, dim, p.size))
    rc = _load().ffo_tangent(rhs_id, method, dim, P, _ptr(x0), _ptr(p), p.size, pparam_index, _ptr(pp), _ptr(hh),
                             int(n_steps), _ptr(xT), _ptr(S), _ptr(Q))
    if rc != 0:
        raise ValueError("ffo_tangent: bad arguments or system without derivatives")
    return xT, S, Q


def mse_gradients(rhs_id, x0, params, h, n_steps, target, pparam_index=-1, pparam=None, method=RK4):
    """Loss L = (1/P) sum_i |x_i(T) - t_i|^2 and its gradients from the forward sensitivities:
    dL/dx0 [dim][P] and dL/dp [n_params] (with a per-particle parameter, its column is summed)."""
    xT, S, Q = tangent(rhs_id, x0, params, h, n_steps, pparam_index, pparam, method)
    P = xT.shape[1]
    r = xT - target
    L = float((r * r).sum() / P)
    g = (2.0 / P) * r
    dx0 = np.einsum("pij,ip->jp", S, g)
    dp = np.einsum("piq,ip->q", Q, g)
    return L, dx0, dp


def count_escaped(state):
    """Number of escaped particles (non-finite or |x| > 1e30) and their flags."""
    st = _c(state, np.float64)
    dim, P = st.shape
    flags = np.zeros(P, dtype=np.uint8)
    n = _load().ffo_count_escaped(dim, P, P, _ptr(st), _ptr(flags))
    return int(n), flags.astype(bool)


def splat2d(u, v, lo, hi, W, H, include=None, image=None):
    """FP32 2D projection + count splat; returns uint32 image [H][W]."""
    u = _c(u, np.float32)
    v = _c(v, np.float32)
    inc = None if include is None else _c(include, np.uint8)
    img = np.zeros((H, W), dtype=np.uint32) if image is None else image
    _load().ffo_splat2d(u.size, _ptr(u), _ptr(v), _ptr(inc), float(lo[0]), float(hi[0]),
                        float(lo[1]), float(hi[1]), W, H, _ptr(img))
    return img


def splat3d(x, y, z, mvp, W, H, include=None, image=None):
    """FP32 3D perspective projection + count splat; mvp column-major 16 floats."""
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    z = _c(z, np.float32)
    m = _c(mvp, np.float32).reshape(16)
    inc = None if include is None else _c(include, np.uint8)
    img = np.zeros((H, W), dtype=np.uint32) if image is None else image
    _load().ffo_splat3d(x.size, _ptr(x), _ptr(y), _ptr(z), _ptr(inc), _ptr(m), W, H, _ptr(img))
    return img


def _sprite_buffers(W, H, group, colour, P):
    g = np.zeros(P, np.int32) if group is None else _c(group, np.int32)
    col = _c(colour, np.float64).reshape(-1, 4)
    if g.size and (g.min() < 0 or g.max() >= col.shape[0]):
        raise ValueError("group index without a colour")
    return g, col, np.zeros((H, W, 4)), np.zeros((H, W, 4)), np.zeros((H, W), np.uint32)


def sprites2d(u, v, lo, hi, W, H, radius, gain, colour, group=None, include=None):
    """Soft sprites of a 2D view: returns (image [H][W][4], sum of |contributions|
    per channel [H][W][4], fragments per pixel [H][W]), all from FP64 sums."""
    u = _c(u, np.float32)
    v = _c(v, np.float32)
    g, col, img, aimg, frags = _sprite_buffers(W, H, group, colour, u.size)
    inc = None if include is None else _c(include, np.uint8)
    _load().ffo_sprites2d(u.size, _ptr(u), _ptr(v), _ptr(g), _ptr(inc), float(lo[0]), float(hi[0]), float(lo[1]),
                          float(hi[1]), W, H, float(radius), float(gain), _ptr(col), _ptr(img), _ptr(aimg),
                          _ptr(frags))
    return img, aimg, frags


def sprites3d(x, y, z, mvp, W, H, radius, gain, colour, group=None, include=None):
    """Soft sprites of a 3D perspective view (constant on-screen size)."""
    x = _c(x, np.float32)
    y = _c(y, np.float32)
    z = _c(z, np.float32)
    m = _c(mvp, np.float32).reshape(16)
    g, col, img, aimg, frags = _sprite_buffers(W, H, group, colour, x.size)
    inc = None if include is None else _c(include, np.uint8)
    _load().ffo_sprites3d(x.size, _ptr(x), _ptr(y), _ptr(z), _ptr(g), _ptr(inc), _ptr(m), W, H, float(radius),
                          float(gain), _ptr(col), _ptr(img), _ptr(aimg), _ptr(frags))
    return img, aimg, frags

