"""Thin ctypes binding of libsrn (include/srn.h).

Each function has the name of its C entry point and only marshals arguments:
device pointers are passed as integers (e.g. ``tensor.data_ptr()``), streams as
integers (``torch.cuda.Stream.cuda_stream``), host arrays as Python sequences.
A non-OK status raises :class:`SrnError` with the library's message.  Nothing
here computes any part of the model; if libsrn.so is missing, loading fails
loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as ct
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsrn.so")

SRN_OK = 0
SRN_ERR_INVALID_ARG = 1
SRN_ERR_UNSUPPORTED = 2
SRN_ERR_CUDA = 3
SRN_ERR_DEVICE_TIMEOUT = 4
SRN_ERR_NONFINITE = 5
SRN_ERR_STATE = 6
SRN_FP32 = 0
SRN_BF16 = 1
SRN_DENSITY = 1
SRN_UPSTREAM = 2
SRN_SCHEDULE = 4
SRN_REC_DG = 8
SRN_VOLUME_TILED = 16
SRN_MAX_BRICKS = 64

# Every symbol include/srn.h declares (checked by the CPU tests).
EXPORTS = (
    "srn_param_layout", "srn_workspace_size", "srn_create", "srn_destroy", "srn_last_error",
    "srn_sync_shadow", "srn_sample_points", "srn_sample_target", "srn_forward", "srn_backward",
    "srn_step", "srn_train_step", "srn_render", "srn_set_timing", "srn_read_timing", "srn_get_status",
    "srn_sample_points_static", "srn_decode", "srn_state_bytes", "srn_save_state", "srn_load_state",
    "srn_set_schedule", "srn_read_schedule", "srn_render_progressive", "srn_get_tuning", "srn_set_tuning",
    "srn_autotune", "srn_rebalance", "srn_tiled_volume_bytes", "srn_tile_volume", "srn_sample_target_tiled",
)
SRN_STATIC_SAMPLER_MAX_POINTS = 131072
SRN_STATIC_SAMPLER_MAX_BRICKS = 8


class SrnError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libsrn status {status}: {message}")
        self.status = status


class Config(ct.Structure):
    _fields_ = [("n_bricks", ct.c_int32), ("n_grids", ct.c_int32), ("channels", ct.c_int32),
                ("res", ct.c_int32), ("hidden", ct.c_int32), ("precision", ct.c_int32),
                ("flat_top_p", ct.c_int32), ("density_eps", ct.c_float), ("lr_feat", ct.c_float),
                ("lr_xform", ct.c_float), ("beta1", ct.c_float), ("beta2", ct.c_float),
                ("adam_eps", ct.c_float)]


class Schedule(ct.Structure):
    _fields_ = [("delay_iters", ct.c_int32), ("density_window", ct.c_int32), ("density_rel", ct.c_float),
                ("density_frac", ct.c_float), ("total_iters", ct.c_int64), ("plateau_window", ct.c_int32),
                ("plateau_rel", ct.c_float), ("plateau_factor", ct.c_float), ("plateau_max", ct.c_int32)]


class BrickSchedule(ct.Structure):
    _fields_ = [("iteration", ct.c_int64), ("lr_scale", ct.c_float), ("plateaus", ct.c_int32),
                ("finished", ct.c_int32), ("density_on", ct.c_int32), ("density_stopped", ct.c_int32),
                ("density_iters", ct.c_int32), ("best_rec", ct.c_double)]


class Tuning(ct.Structure):
    _fields_ = [("tile_points", ct.c_int32), ("tile_level", ct.c_int32), ("density_ctas", ct.c_int32)]


class Layout(ct.Structure):
    _fields_ = [(n, ct.c_int64) for n in (
        "n_params", "n_group_a", "off_F", "off_W1", "off_W2", "off_w3", "off_G",
        "size_F", "size_W1", "size_W2", "size_w3", "size_G")]


class Tensors(ct.Structure):
    _fields_ = [("params_dev", ct.c_void_p), ("grads_dev", ct.c_void_p), ("adam_m_dev", ct.c_void_p),
                ("adam_v_dev", ct.c_void_p), ("shadow_dev", ct.c_void_p), ("range_dev", ct.c_void_p)]


class Camera(ct.Structure):
    _fields_ = [("eye", ct.c_float * 3), ("forward", ct.c_float * 3), ("right", ct.c_float * 3),
                ("up", ct.c_float * 3), ("scale", ct.c_float), ("ortho", ct.c_int32)]


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Load libsrn.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2308_02494_gb300.build`")
    lib = ct.CDLL(path)
    P, I64, I32, U64, U32, F = ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_uint64, ct.c_uint32, ct.c_float
    I64P = ct.POINTER(ct.c_int64)
    sig = {
        "srn_param_layout": [ct.POINTER(Config), ct.POINTER(Layout)],
        "srn_workspace_size": [ct.POINTER(Config), I64, ct.POINTER(ct.c_size_t)],
        "srn_create": [ct.POINTER(Config), ct.POINTER(Tensors), P, ct.c_size_t, I64, ct.POINTER(P)],
        "srn_destroy": [P],
        "srn_sync_shadow": [P, P],
        "srn_sample_points": [P, P, U64, U64, P, I64P, P],
        "srn_sample_target": [P, P, P, I64P, I64P, P, I64P, P],
        "srn_sample_target_tiled": [P, P, P, I64P, I64P, P, I64P, P],
        "srn_tiled_volume_bytes": [I64P, ct.POINTER(ct.c_size_t)],
        "srn_tile_volume": [P, P, I64P, P],
        "srn_forward": [P, P, P, I64P, P],
        "srn_backward": [P, P, P, P, I64P, U32, P],
        "srn_step": [P, P, U32],
        "srn_train_step": [P, P, U64, P, I64P, I64P, I64P, U32, P, P, P],
        "srn_render": [P, P, ct.POINTER(Camera), P, F, F, I32, I32, I32, ct.POINTER(I32), I64P, I64, P],
        "srn_render_progressive": [P, P, ct.POINTER(Camera), P, F, F, I32, I32, I32, ct.POINTER(I32), I64P, I64,
                                   I64, I64, P, P],
        "srn_get_status": [P, P],
        "srn_set_timing": [P, I32],
        "srn_read_timing": [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64)],
        "srn_sample_points_static": [P, U64, U64, I32, I64P, P],
        "srn_decode": [P, P, ct.POINTER(ct.c_int32), I64P, I64, P],
        "srn_state_bytes": [P, ct.POINTER(ct.c_size_t)],
        "srn_set_schedule": [P, ct.POINTER(Schedule)],
        "srn_read_schedule": [P, P, ct.POINTER(BrickSchedule)],
        "srn_save_state": [P, P, P, ct.c_size_t],
        "srn_load_state": [P, P, P, ct.c_size_t],
        "srn_get_tuning": [P, ct.POINTER(Tuning)],
        "srn_set_tuning": [P, ct.POINTER(Tuning)],
        "srn_autotune": [P, P, P, P, I64P, U32, I32, ct.POINTER(Tuning)],
        "srn_rebalance": [I32, I64P, ct.POINTER(BrickSchedule), I64, I64P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ct.c_int
    lib.srn_last_error.argtypes = []
    lib.srn_last_error.restype = ct.c_char_p
    _lib = lib
    return lib


def _check(st: int) -> None:
    if st != SRN_OK:
        raise SrnError(st, load().srn_last_error().decode())


def _i64(seq) -> ct.Array:
    vals = [int(v) for v in seq]
    return (ct.c_int64 * len(vals))(*vals)


def srn_last_error() -> str:
    return load().srn_last_error().decode()


def srn_param_layout(cfg: Config) -> Layout:
    out = Layout()
    _check(load().srn_param_layout(ct.byref(cfg), ct.byref(out)))
    return out


def srn_workspace_size(cfg: Config, max_points: int) -> int:
    n = ct.c_size_t()
    _check(load().srn_workspace_size(ct.byref(cfg), max_points, ct.byref(n)))
    return n.value


def srn_create(cfg: Config, tensors: Tensors, workspace: int, workspace_bytes: int, max_points: int) -> int:
    h = ct.c_void_p()
    _check(load().srn_create(ct.byref(cfg), ct.byref(tensors), workspace, workspace_bytes,
                             max_points, ct.byref(h)))
    return h.value


def srn_destroy(h: int) -> None:
    _check(load().srn_destroy(h))


def srn_sync_shadow(h: int, stream: int) -> None:
    _check(load().srn_sync_shadow(h, stream))


def srn_sample_points(h, stream, seed, step, step_dev, offsets, xyz) -> None:
    _check(load().srn_sample_points(h, stream, seed, step, step_dev, _i64(offsets), xyz))


def srn_sample_target(h, stream, volume, dims, boxes, xyz, offsets, target) -> None:
    _check(load().srn_sample_target(h, stream, volume, _i64(dims), _i64(boxes), xyz, _i64(offsets), target))


def srn_sample_target_tiled(h, stream, tiled, dims, boxes, xyz, offsets, target) -> None:
    _check(load().srn_sample_target_tiled(h, stream, tiled, _i64(dims), _i64(boxes), xyz, _i64(offsets), target))


def srn_tiled_volume_bytes(dims) -> int:
    n = ct.c_size_t()
    _check(load().srn_tiled_volume_bytes(_i64(dims), ct.byref(n)))
    return n.value


def srn_tile_volume(stream, volume, dims, tiled) -> None:
    _check(load().srn_tile_volume(stream, volume, _i64(dims), tiled))


def srn_forward(h, stream, xyz, offsets, out) -> None:
    _check(load().srn_forward(h, stream, xyz, _i64(offsets), out))


def srn_backward(h, stream, xyz, target, offsets, flags, losses) -> None:
    _check(load().srn_backward(h, stream, xyz, target, _i64(offsets), flags, losses))


def srn_step(h, stream, flags) -> None:
    _check(load().srn_step(h, stream, flags))


def srn_train_step(h, stream, seed, volume, dims, boxes, offsets, flags, xyz, target, losses) -> None:
    _check(load().srn_train_step(h, stream, seed, volume, _i64(dims), _i64(boxes), _i64(offsets),
                                 flags, xyz, target, losses))


def srn_render(h, stream, cam: Camera, lut, vmin, vmax, width, height, samples, grid, boxes, vox, rgba) -> None:
    g = (ct.c_int32 * 3)(*[int(v) for v in grid])
    _check(load().srn_render(h, stream, ct.byref(cam), lut, vmin, vmax, width, height, samples, g,
                             _i64(boxes), vox, rgba))


def srn_render_progressive(h, stream, cam: Camera, lut, vmin, vmax, width, height, samples, grid, boxes, vox,
                           first, count, rgba, preview) -> None:
    g = (ct.c_int32 * 3)(*[int(v) for v in grid])
    _check(load().srn_render_progressive(h, stream, ct.byref(cam), lut, vmin, vmax, width, height, samples, g,
                                         _i64(boxes), vox, int(first), int(count), rgba, preview))


SRN_TIME_OFF, SRN_TIME_QUERY, SRN_TIME_ENCODER, SRN_TIME_DECODER, SRN_TIME_SCATTER = range(5)


def srn_set_timing(h, target) -> None:
    """target: SRN_TIME_* (True means SRN_TIME_QUERY, False SRN_TIME_OFF)."""
    _check(load().srn_set_timing(h, int(target)))


def srn_read_timing(h) -> tuple:
    ms, n = ct.c_double(), ct.c_int64()
    _check(load().srn_read_timing(h, ct.byref(ms), ct.byref(n)))
    return ms.value, n.value


def srn_sample_points_static(stream, seed, step, n_bricks, offsets, xyz) -> None:
    """Batch sampler that allocates nothing (scratch in a static device array)."""
    _check(load().srn_sample_points_static(stream, seed, step, n_bricks, _i64(offsets), xyz))


def srn_decode(h, stream, grid, boxes, vox, out) -> None:
    g = (ct.c_int32 * 3)(*[int(v) for v in grid])
    _check(load().srn_decode(h, stream, g, _i64(boxes), int(vox), out))


def srn_set_schedule(h, sched: Schedule) -> None:
    _check(load().srn_set_schedule(h, ct.byref(sched)))


def srn_read_schedule(h, stream, n_bricks: int) -> list:
    out = (BrickSchedule * n_bricks)()
    _check(load().srn_read_schedule(h, stream, out))
    return [{f: getattr(o, f) for f, _ in BrickSchedule._fields_} for o in out]


def srn_rebalance(base_counts, finished, min_points) -> list:
    """Batch offsets after bricks finish; `finished` is one flag per brick (or
    srn_read_schedule's dicts)."""
    n = len(base_counts)
    st = (BrickSchedule * n)()
    for b, f in enumerate(finished):
        st[b].finished = int(f["finished"] if isinstance(f, dict) else f)
    out = (ct.c_int64 * (n + 1))()
    _check(load().srn_rebalance(n, _i64(base_counts), st, int(min_points), out))
    return list(out)


def srn_state_bytes(h) -> int:
    n = ct.c_size_t()
    _check(load().srn_state_bytes(h, ct.byref(n)))
    return n.value


def srn_save_state(h, stream) -> bytes:
    n = srn_state_bytes(h)
    buf = (ct.c_ubyte * n)()
    _check(load().srn_save_state(h, stream, buf, n))
    return bytes(buf)


def srn_load_state(h, stream, blob: bytes) -> None:
    buf = (ct.c_ubyte * len(blob)).from_buffer_copy(blob)
    _check(load().srn_load_state(h, stream, buf, len(blob)))


def srn_get_tuning(h) -> dict:
    out = Tuning()
    _check(load().srn_get_tuning(h, ct.byref(out)))
    return {f: getattr(out, f) for f, _ in Tuning._fields_}


def srn_set_tuning(h, tile_points, tile_level, density_ctas) -> None:
    _check(load().srn_set_tuning(h, ct.byref(Tuning(tile_points, tile_level, density_ctas))))


def srn_autotune(h, stream, xyz, target, offsets, flags, reps) -> dict:
    out = Tuning()
    _check(load().srn_autotune(h, stream, xyz, target, _i64(offsets), flags, reps, ct.byref(out)))
    return {f: getattr(out, f) for f, _ in Tuning._fields_}


def srn_get_status(h, stream) -> None:
    _check(load().srn_get_status(h, stream))
