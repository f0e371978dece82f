"""GB300-native Fireflies hot path: ctypes binding of ``libff.so`` (include/ff.h).

Argument marshalling only -- every step of the path (seeding, integration,
projection, splatting, statistics) runs in the CUDA kernels of ``libff.so``.
There is no CPU fallback: if the library is not built or cannot be loaded,
every call raises.

Functions carry the C names (``ff_create_system``, ``ff_seed_particles``,
``ff_step``, ``ff_set_params``, ``ff_project_splat``, ...).  Buffers may be
torch CUDA tensors (device), numpy arrays (host) or raw integer device
pointers.  ``System`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads  # noqa: F401  (inputs only; no arithmetic of the method)

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libff.so")

FF_OK, FF_ERR_INVALID_ARG, FF_ERR_CUDA, FF_ERR_OOM, FF_ERR_STATE, FF_ERR_UNSUPPORTED, FF_ERR_TIMEOUT = range(7)
FF_RHS_LINEAR, FF_RHS_HARMONIC, FF_RHS_WILSON_COWAN, FF_RHS_LORENZ, FF_RHS_HH3 = range(5)
FF_RK4, FF_EULER = 0, 1
FF_FLAG_KAHAN = 1
FF_MAX_DIM, FF_MAX_PARAMS, FF_MAX_GROUPS = 16, 64, 16

RHS_BY_NAME = {"linear": FF_RHS_LINEAR, "harmonic": FF_RHS_HARMONIC, "wilson_cowan": FF_RHS_WILSON_COWAN,
               "lorenz": FF_RHS_LORENZ, "hh3": FF_RHS_HH3}
METHOD_BY_NAME = {"rk4": FF_RK4, "euler": FF_EULER}


class FFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"[ff status {status}] {message}")
        self.status = status


class ff_view(ctypes.Structure):
    _fields_ = [("ndim_view", ctypes.c_int), ("axes", ctypes.c_int * 3), ("lo", ctypes.c_double * 2),
                ("hi", ctypes.c_double * 2), ("mvp", ctypes.c_float * 16), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("group_mask", ctypes.c_uint32), ("accumulate", ctypes.c_int)]


FF_SPRITE_AUTO, FF_SPRITE_DIRECT, FF_SPRITE_TILED = 0, 1, 2


class ff_sprite(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_float), ("gain", ctypes.c_float),
                ("colour", (ctypes.c_float * 4) * FF_MAX_GROUPS), ("technique", ctypes.c_int)]


def make_sprite(radius=1.5, gain=1.0, colours=((1.0, 1.0, 1.0, 1.0),), technique=FF_SPRITE_AUTO):
    """A soft-sprite description: radius in pixels, gain, up to FF_MAX_GROUPS rows of
    4 channel weights (groups beyond the rows given get zeros) and the summation
    technique (FF_SPRITE_AUTO / DIRECT / TILED)."""
    sp = ff_sprite()
    sp.radius = float(radius)
    sp.gain = float(gain)
    sp.technique = int(technique)
    rows = np.asarray(colours, dtype=np.float64).reshape(-1, 4)
    if rows.shape[0] > FF_MAX_GROUPS:
        raise ValueError(f"at most {FF_MAX_GROUPS} colour rows")
    for g, row in enumerate(rows):
        for k in range(4):
            sp.colour[g][k] = float(row[k])
    return sp


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "ff_create_system": [ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_uint, _I64, _P,
                         ctypes.POINTER(_P)],
    "ff_destroy_system": [_P],
    "ff_seed_particles": [_P, _I64, _P, _P, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)],
    "ff_seed_particles_slice": [_P, _I64, _I64, _I64, _P, _P, ctypes.c_int, ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_int)],
    "ff_set_particle_param_slice": [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _I64, _I64],
    "ff_reset": [_P],
    "ff_set_particle_param": [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double],
    "ff_set_particle_param_values": [_P, ctypes.c_int, _P, ctypes.c_int],
    "ff_get_particle_param": [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "ff_step": [_P, _I64, ctypes.c_double],
    "ff_set_params": [_P, _P, ctypes.c_int],
    "ff_project_splat": [_P, ctypes.POINTER(ff_view), _P, ctypes.c_int],
    "ff_step_splat": [_P, _I64, ctypes.c_double, ctypes.POINTER(ff_view), _P, ctypes.c_int],
    "ff_project_sprites": [_P, ctypes.POINTER(ff_view), ctypes.POINTER(ff_sprite), _P, ctypes.c_int],
    "ff_get_state": [_P, _P, ctypes.c_int],
    "ff_set_state": [_P, _P, ctypes.c_int],
    "ff_stats": [_P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "ff_system_info": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int)],
    "ff_set_launch": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I64],
    "ff_last_launch": [_P, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "ff_backward": [_P, _P, _P, _P],
    "ff_count_escaped_noalloc": [_P, ctypes.c_int, _I64, _I64, _P, ctypes.c_int, _P, _P],
    "ff_pipe_rate": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "ff_set_reset": [_P, _P, _P, ctypes.c_double, ctypes.c_int],
    "ff_tape_begin": [_P, _I64, _I64],
    "ff_batch_create": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
    "ff_batch_step": [_P, _I64, _P],
    "ff_batch_autotune": [_P, _P, _I64],
    "ff_batch_describe": [_P, ctypes.c_char_p, ctypes.c_int],
    "ff_batch_destroy": [_P],
    "ff_batch_tape_begin": [_P, _I64, _I64],
    "ff_batch_tape_end": [_P],
    "ff_batch_backward": [_P, _P, _P, _P],
    "ff_tape_end": [_P],
    "ff_get_reset_state": [_P, _P, _P, ctypes.c_int],
}


def lib():
    """The loaded ``libff.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                               "(or python -m paper_1505_00344_gb300._build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.ff_last_error.argtypes = []
        L.ff_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != FF_OK:
        raise FFError(status, lib().ff_last_error().decode(errors="replace"))


def _buf(obj, dtype=None, min_elems=0):
    """(pointer, is_device, keepalive) of a torch tensor, numpy array or int device pointer.

    With ``dtype`` the array or tensor must hold that element type (a uint32 buffer
    may also be an int32 tensor, as torch images usually are); with ``min_elems``
    it must hold at least that many elements.  A raw int pointer is taken as is.
    """
    if obj is None:
        return None, 0, None
    if isinstance(obj, int):
        return obj, 1, None
    if isinstance(obj, np.ndarray):
        if not obj.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous")
        if dtype is not None and obj.dtype != dtype:
            raise ValueError(f"expected dtype {np.dtype(dtype).name}, got {obj.dtype}")
        if obj.size < min_elems:
            raise ValueError(f"buffer holds {obj.size} elements, the call needs {min_elems}")
        return obj.ctypes.data, 0, obj
    # torch tensor (duck-typed so torch stays optional for host-only callers)
    if hasattr(obj, "data_ptr") and hasattr(obj, "is_cuda"):
        if not obj.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if dtype is not None:
            want = np.dtype(dtype).name
            got = str(obj.dtype).replace("torch.", "")
            if got != want and not (want == "uint32" and got == "int32"):
                raise ValueError(f"expected dtype {want}, got {got}")
        if obj.numel() < min_elems:
            raise ValueError(f"buffer holds {obj.numel()} elements, the call needs {min_elems}")
        return obj.data_ptr(), 1 if obj.is_cuda else 0, obj
    raise TypeError(f"unsupported buffer type {type(obj)}")


def _image_buf(image, view, channels=1, dtype=None):
    """_buf of an image of view.width x view.height x channels 4-byte elements
    (counts: uint32 or int32; sprites: float32)."""
    need = max(int(view.width), 0) * max(int(view.height), 0) * channels
    if dtype is None and isinstance(image, np.ndarray) and image.dtype not in (np.uint32, np.int32):
        raise ValueError(f"count images are uint32 or int32, got {image.dtype}")
    if dtype is None and hasattr(image, "element_size") and not isinstance(image, np.ndarray):
        if str(image.dtype).replace("torch.", "") not in ("int32", "uint32"):
            raise ValueError(f"count images are uint32 or int32, got {image.dtype}")
    return _buf(image, dtype, min_elems=need)


def _state_elems(sys):
    n, _, dim, _ = ff_system_info(sys)
    return n * dim


def _dbl(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
    return a, a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


def ff_create_system(rhs_id, dim, params, method=FF_RK4, flags=0, capacity=1, stream=None):
    p, pp = _dbl(params)
    out = _P()
    _check(lib().ff_create_system(int(rhs_id), int(dim), pp, p.size, int(method), int(flags), int(capacity),
                                  _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def ff_destroy_system(sys):
    _check(lib().ff_destroy_system(sys))


def ff_seed_particles(sys, count, lo, hi, direction, seed):
    lo_a, lo_p = _dbl(lo)
    hi_a, hi_p = _dbl(hi)
    gid = ctypes.c_int(-1)
    _check(lib().ff_seed_particles(sys, int(count), lo_p, hi_p, int(direction), int(seed) & (2**64 - 1),
                                   ctypes.byref(gid)))
    return gid.value


def ff_seed_particles_slice(sys, count, first, total, lo, hi, direction, seed):
    """Particles first .. first + count - 1 of a group of `total` (one GPU's share)."""
    lo_a, lo_p = _dbl(lo)
    hi_a, hi_p = _dbl(hi)
    gid = ctypes.c_int(-1)
    _check(lib().ff_seed_particles_slice(sys, int(count), int(first), int(total), lo_p, hi_p, int(direction),
                                         int(seed) & (2**64 - 1), ctypes.byref(gid)))
    return gid.value


def ff_set_particle_param_slice(sys, param_index, lo, hi, first, total):
    _check(lib().ff_set_particle_param_slice(sys, int(param_index), float(lo), float(hi), int(first), int(total)))


def ff_reset(sys):
    _check(lib().ff_reset(sys))


def ff_set_particle_param(sys, param_index, lo=0.0, hi=0.0):
    _check(lib().ff_set_particle_param(sys, int(param_index), float(lo), float(hi)))


def ff_set_particle_param_values(sys, param_index, values):
    ptr, dev, _keep = _buf(values, np.float32)
    _check(lib().ff_set_particle_param_values(sys, int(param_index), ptr, dev))


def ff_get_particle_param(sys, dst):
    ptr, dev, _keep = _buf(dst, np.float32)
    idx = ctypes.c_int(-1)
    _check(lib().ff_get_particle_param(sys, ptr, dev, ctypes.byref(idx)))
    return idx.value


def ff_set_reset(sys, bound_lo=None, bound_hi=None, t_max=0.0, check_every=1):
    lo = hi = None
    lo_p = hi_p = None
    if bound_lo is not None:
        lo, lo_p = _dbl(bound_lo)
    if bound_hi is not None:
        hi, hi_p = _dbl(bound_hi)
    _check(lib().ff_set_reset(sys, lo_p, hi_p, float(t_max), int(check_every)))


def ff_get_reset_state(sys, age=None, resets=None):
    a, dev_a, _ka = _buf(age, np.uint32)
    r, dev_r, _kr = _buf(resets, np.uint32)
    dev = dev_a if age is not None else dev_r
    _check(lib().ff_get_reset_state(sys, a, r, dev))


def ff_step(sys, n_steps, dt):
    _check(lib().ff_step(sys, int(n_steps), float(dt)))


def ff_set_params(sys, params):
    p, pp = _dbl(params)
    _check(lib().ff_set_params(sys, pp, p.size))


def make_view(ndim_view=2, axes=(0, 1), lo=(0.0, 0.0), hi=(1.0, 1.0), mvp=None, width=256, height=256,
              group_mask=0xFFFFFFFF, accumulate=0, **_ignored):
    v = ff_view()
    v.ndim_view = int(ndim_view)
    ax = list(axes) + [0] * (3 - len(axes))
    for q in range(3):
        v.axes[q] = int(ax[q])
    if ndim_view == 2:
        for q in range(2):
            v.lo[q] = float(lo[q])
            v.hi[q] = float(hi[q])
    m = np.eye(4, dtype=np.float32).reshape(16) if mvp is None else np.asarray(mvp, np.float32).reshape(16)
    for q in range(16):
        v.mvp[q] = float(m[q])
    v.width, v.height = int(width), int(height)
    v.group_mask = int(group_mask) & 0xFFFFFFFF
    v.accumulate = int(accumulate)
    return v


def ff_project_splat(sys, view, image):
    if isinstance(view, dict):
        view = make_view(**view)
    ptr, dev, _keep = _image_buf(image, view)
    _check(lib().ff_project_splat(sys, ctypes.byref(view), ptr, dev))


def ff_step_splat(sys, n_steps, dt, view, image):
    if isinstance(view, dict):
        view = make_view(**view)
    ptr, dev, _keep = _image_buf(image, view)
    _check(lib().ff_step_splat(sys, int(n_steps), float(dt), ctypes.byref(view), ptr, dev))


def ff_project_sprites(sys, view, sprite, image):
    """Soft sprites into a float32 image [height][width][4] (host array or CUDA tensor)."""
    if isinstance(view, dict):
        view = make_view(**view)
    if isinstance(sprite, dict):
        sprite = make_sprite(**sprite)
    ptr, dev, _keep = _image_buf(image, view, channels=4, dtype=np.float32)
    _check(lib().ff_project_sprites(sys, ctypes.byref(view), ctypes.byref(sprite), ptr, dev))


def ff_get_state(sys, dst):
    ptr, dev, _keep = _buf(dst, np.float32, min_elems=_state_elems(sys))
    _check(lib().ff_get_state(sys, ptr, dev))


def ff_set_state(sys, src):
    ptr, dev, _keep = _buf(src, np.float32, min_elems=_state_elems(sys))
    _check(lib().ff_set_state(sys, ptr, dev))


def ff_stats(sys):
    n = _I64(0)
    tf = ctypes.c_double(0)
    tb = ctypes.c_double(0)
    _check(lib().ff_stats(sys, ctypes.byref(n), ctypes.byref(tf), ctypes.byref(tb)))
    return n.value, tf.value, tb.value


def ff_system_info(sys):
    n = _I64(0)
    pitch = _I64(0)
    dim = ctypes.c_int(0)
    ng = ctypes.c_int(0)
    _check(lib().ff_system_info(sys, ctypes.byref(n), ctypes.byref(pitch), ctypes.byref(dim), ctypes.byref(ng)))
    return n.value, pitch.value, dim.value, ng.value


def ff_last_launch(sys):
    """What the last ff_step / ff_step_splat launched: dict with the integrator kernel's
    name, grid, block, whether the splat was fused into it, and the launch counts."""
    buf = ctypes.create_string_buffer(512)
    grid, block, fused = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    n_int, n_splat = _I64(0), _I64(0)
    _check(lib().ff_last_launch(sys, buf, len(buf), ctypes.byref(grid), ctypes.byref(block), ctypes.byref(fused),
                                ctypes.byref(n_int), ctypes.byref(n_splat)))
    return {"kernel": buf.value.decode(), "grid": grid.value, "block": block.value, "fused_splat": bool(fused.value),
            "integrator_launches": n_int.value, "splat_launches": n_splat.value}


def ff_set_launch(sys, particles_per_thread=1, block=256, blocks_per_sm=0, max_steps_per_launch=0):
    _check(lib().ff_set_launch(sys, int(particles_per_thread), int(block), int(blocks_per_sm),
                               int(max_steps_per_launch)))


def ff_tape_begin(sys, checkpoint_every=100, max_steps=1):
    _check(lib().ff_tape_begin(sys, int(checkpoint_every), int(max_steps)))


def ff_tape_end(sys):
    _check(lib().ff_tape_end(sys))


def ff_backward(sys, dL_dxT, dL_dx0, dL_dp=None):
    """Reverse sweep: dL_dxT / dL_dx0 device buffers [dim][P]; returns dL/dp (host float64)."""
    a, dev_a, _ka = _buf(dL_dxT)
    b, dev_b, _kb = _buf(dL_dx0)
    if not (dev_a and dev_b):
        raise ValueError("dL_dxT and dL_dx0 must be device buffers")
    n_params = ctypes.c_int(0)
    if dL_dp is None:
        dL_dp = np.zeros(FF_MAX_PARAMS, np.float64)
    if dL_dp.size < FF_MAX_PARAMS:
        raise ValueError(f"dL_dp needs room for FF_MAX_PARAMS = {FF_MAX_PARAMS} doubles")
    c, _, _kc = _buf(dL_dp, np.float64)
    _check(lib().ff_backward(sys, a, b, c))
    return dL_dp


FF_NOALLOC_MAX_GROUPS = 256
FF_PIPE_FFMA, FF_PIPE_FFMA2, FF_PIPE_EX2, FF_PIPE_RCP, FF_PIPE_LOGISTIC = range(5)


def ff_pipe_rate(op, device=0):
    """Measured lane operations per second of one instruction kind (FF_PIPE_*) on a device."""
    out = ctypes.c_double(0.0)
    _check(lib().ff_pipe_rate(int(op), int(device), ctypes.byref(out)))
    return out.value


def ff_count_escaped_noalloc(state, dim, n_particles, pitch, group_starts, stream=None):
    """Escaped particles per group of a device SoA state, without any device allocation.

    For callers that must not allocate device memory at call time (see
    include/ff.h); ``state`` is a device buffer (float32 tensor or pointer) of at
    least (dim - 1) * pitch + n_particles floats, the result a host int64 array
    with one count per group.  A tensor of another dtype or too few elements is
    rejected here, before anything reaches the GPU.
    """
    dim, n_particles, pitch = int(dim), int(n_particles), int(pitch)
    if dim < 1 or n_particles < 0 or pitch < n_particles:
        raise ValueError("dim must be >= 1 and 0 <= n_particles <= pitch")
    need = (dim - 1) * pitch + n_particles if n_particles > 0 else 0
    ptr, dev, _keep = _buf(state, np.float32, min_elems=need)
    if not dev:
        raise ValueError("state must be device memory")
    starts = np.ascontiguousarray(np.asarray(group_starts, dtype=np.int64).reshape(-1))
    counts = np.zeros(starts.size, dtype=np.int64)
    _check(lib().ff_count_escaped_noalloc(ptr, dim, n_particles, pitch, starts.ctypes.data,
                                          starts.size, _stream_ptr(stream), counts.ctypes.data))
    return counts


def ff_batch_create(systems, stream=None):
    """systems: ff_system handles (or System objects)."""
    handles = [getattr(x, "handle", x) for x in systems]
    arr = (_P * len(handles))(*handles)
    out = _P()
    _check(lib().ff_batch_create(arr, len(handles), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def ff_batch_step(batch, n_steps, dt):
    d, dp = _dbl(dt)
    _check(lib().ff_batch_step(batch, int(n_steps), dp))


def ff_batch_autotune(batch, dt, trial_steps=64):
    d, dp = _dbl(dt)
    _check(lib().ff_batch_autotune(batch, dp, int(trial_steps)))


def ff_batch_describe(batch):
    buf = ctypes.create_string_buffer(4096)
    _check(lib().ff_batch_describe(batch, buf, len(buf)))
    return buf.value.decode()


def ff_batch_destroy(batch):
    _check(lib().ff_batch_destroy(batch))


def ff_batch_tape_begin(batch, checkpoint_every, max_steps):
    _check(lib().ff_batch_tape_begin(batch, int(checkpoint_every), int(max_steps)))


def ff_batch_tape_end(batch):
    _check(lib().ff_batch_tape_end(batch))


def ff_batch_backward(batch, dL_dxT, dL_dx0):
    """dL_dxT, dL_dx0: one CUDA tensor (or device pointer) per member, SoA [dim][P].
    Returns the parameter gradients, an array [n_systems][FF_MAX_PARAMS] (float64)."""
    if len(dL_dxT) != len(dL_dx0):
        raise ValueError("one input and one output buffer per member")
    n = len(dL_dxT)
    ins = (ctypes.c_void_p * n)(*[_buf(t)[0] for t in dL_dxT])
    outs = (ctypes.c_void_p * n)(*[_buf(t)[0] for t in dL_dx0])
    for t in list(dL_dxT) + list(dL_dx0):
        if _buf(t)[1] != 1:
            raise ValueError("gradient buffers must be device memory")
    dp = np.zeros((n, FF_MAX_PARAMS), np.float64)
    _check(lib().ff_batch_backward(batch, ins, outs, dp.ctypes.data))
    return dp


class Batch:
    """Owning handle over one ff_batch (the systems stay owned by their System objects)."""

    def __init__(self, systems, stream=None):
        self.systems = list(systems)  # keep the systems alive as long as the batch
        self.handle = ff_batch_create(self.systems, stream)

    def step(self, n_steps, dt):
        ff_batch_step(self.handle, n_steps, dt)

    def autotune(self, dt, trial_steps=64):
        ff_batch_autotune(self.handle, dt, trial_steps)

    def describe(self):
        return ff_batch_describe(self.handle)

    def tape_begin(self, checkpoint_every, max_steps):
        ff_batch_tape_begin(self.handle, checkpoint_every, max_steps)

    def tape_end(self):
        ff_batch_tape_end(self.handle)

    def backward(self, dL_dxT, dL_dx0):
        return ff_batch_backward(self.handle, dL_dxT, dL_dx0)

    def close(self):
        if getattr(self, "handle", None):
            ff_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ff_last_error():
    return lib().ff_last_error().decode(errors="replace")


class System:
    """Owning handle over one ``ff_system`` (thin wrapper over the ff_* calls)."""

    def __init__(self, rhs, params, capacity, dim=None, method="rk4", kahan=False, stream=None):
        rhs_id = RHS_BY_NAME[rhs] if isinstance(rhs, str) else int(rhs)
        if dim is None:
            dim = {FF_RHS_HARMONIC: 2, FF_RHS_WILSON_COWAN: 2, FF_RHS_LORENZ: 3, FF_RHS_HH3: 15}.get(rhs_id)
            if dim is None:
                dim = int(round(np.sqrt(len(params))))
        meth = METHOD_BY_NAME[method] if isinstance(method, str) else int(method)
        self.dim = dim
        self.handle = ff_create_system(rhs_id, dim, params, meth, FF_FLAG_KAHAN if kahan else 0, capacity, stream)

    @classmethod
    def from_workload(cls, w, kahan=False, stream=None, capacity=None):
        """Create and seed a system from a ``workloads`` description."""
        total = sum(g["count"] for g in w["groups"])
        s = cls(w["rhs"], w["params"], capacity or total, dim=w["dim"], method=w.get("method", "rk4"),
                kahan=kahan, stream=stream)
        for g in w["groups"]:
            s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
        if "pparam" in w:
            pp = w["pparam"]
            s.set_particle_param(pp["index"], pp["lo"], pp["hi"])
        return s

    def seed(self, count, lo, hi, direction, seed):
        return ff_seed_particles(self.handle, count, lo, hi, direction, seed)

    def seed_slice(self, count, first, total, lo, hi, direction, seed):
        return ff_seed_particles_slice(self.handle, count, first, total, lo, hi, direction, seed)

    def set_particle_param_slice(self, index, lo, hi, first, total):
        ff_set_particle_param_slice(self.handle, index, lo, hi, first, total)

    def reset(self):
        ff_reset(self.handle)

    def set_particle_param(self, index, lo=0.0, hi=0.0):
        ff_set_particle_param(self.handle, index, lo, hi)

    def set_particle_param_values(self, index, values):
        ff_set_particle_param_values(self.handle, index, values)

    def get_particle_param(self, dst):
        return ff_get_particle_param(self.handle, dst)

    def step(self, n_steps, dt):
        ff_step(self.handle, n_steps, dt)

    def tape_begin(self, checkpoint_every=100, max_steps=1):
        ff_tape_begin(self.handle, checkpoint_every, max_steps)

    def tape_end(self):
        ff_tape_end(self.handle)

    def backward(self, dL_dxT, dL_dx0, n_params):
        # the call writes every parameter of the system: hand it room for FF_MAX_PARAMS
        return ff_backward(self.handle, dL_dxT, dL_dx0)[:n_params]

    def set_reset(self, bound_lo=None, bound_hi=None, t_max=0.0, check_every=1):
        ff_set_reset(self.handle, bound_lo, bound_hi, t_max, check_every)

    def get_reset_state(self, age=None, resets=None):
        ff_get_reset_state(self.handle, age, resets)

    def set_params(self, params):
        ff_set_params(self.handle, params)

    def project_splat(self, view, image):
        ff_project_splat(self.handle, view, image)

    def step_splat(self, n_steps, dt, view, image):
        ff_step_splat(self.handle, n_steps, dt, view, image)

    def project_sprites(self, view, sprite, image):
        ff_project_sprites(self.handle, view, sprite, image)

    def get_state(self, dst):
        ff_get_state(self.handle, dst)

    def set_state(self, src):
        ff_set_state(self.handle, src)

    def stats(self):
        return ff_stats(self.handle)

    def info(self):
        return ff_system_info(self.handle)

    def last_launch(self):
        """ff_last_launch: the integrator kernel, shape and fusion of the last step call."""
        return ff_last_launch(self.handle)

    def set_launch(self, particles_per_thread=0, block=0, blocks_per_sm=0, max_steps_per_launch=0):
        """Launch shape (0 keeps the current particles per thread or block size)."""
        ff_set_launch(self.handle, particles_per_thread, block, blocks_per_sm, max_steps_per_launch)

    @property
    def n_particles(self):
        return self.info()[0]

    def close(self):
        if getattr(self, "handle", None):
            ff_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
