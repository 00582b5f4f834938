"""ctypes binding of ``libac.so`` (the C ABI declared in include/ac.h).

Argument marshalling only: every function forwards to the C entry point of
the same name.  Device memory and streams come from PyTorch; the library
receives plain pointers.  There is no fallback: if the CUDA library cannot
be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

AC_OK = 0
AC_ERR_INVALID = 1
AC_ERR_CUDA = 2
AC_ERR_NONFINITE = 3
AC_ERR_TIMEOUT = 4
AC_ERR_UNSUPPORTED = 5
AC_ERR_NOMEM = 6

AC_F64, AC_F32, AC_F16S = 0, 1, 2
AC_VARIANT_AUTO, AC_VARIANT_DIRECT, AC_VARIANT_STREAM = 0, 1, 2
AC_MAX_K = 8
AC_TILE_AUTO, AC_NUM_TILES_3D, AC_NUM_TILES_2D = -1, 3, 2
AC_SHAPE_DUMBBELL, AC_SHAPE_STAR, AC_SHAPE_TORUS = 1, 2, 3

EXPORTED = (
    "ac_workspace_bytes", "ac_create", "ac_step", "ac_energy", "ac_phase_volume", "ac_observe",
    "ac_init_sphere", "ac_init_random", "ac_init_shape", "ac_set_schedule", "ac_get_schedule", "ac_set_tile",
    "ac_get_tile", "ac_autotune", "ac_set_tune_cache",
    "ac_set_graph", "ac_status", "ac_launch_count", "ac_observe_noalloc", "ac_destroy",
    "ac_last_error", "ac_version",
    "ac_batch_workspace_bytes", "ac_batch_create", "ac_batch_step", "ac_batch_set_schedule",
    "ac_batch_get_schedule", "ac_batch_set_tile", "ac_batch_get_tile", "ac_batch_autotune", "ac_batch_set_graph", "ac_batch_observe",
    "ac_batch_status", "ac_batch_set_wait_limit", "ac_batch_launch_count", "ac_batch_destroy",
    "ac_tc_gemm_bf16_n32",
    "ac_net_param_count", "ac_net_create", "ac_net_set_params", "ac_net_get_params",
    "ac_net_forward", "ac_net_loss_grads", "ac_net_adam", "ac_net_train_step",
    "ac_net_launch_count", "ac_net_destroy", "ac_learned_advance", "ac_net_train",
    "ac_net_init_params", "ac_jump_residual", "ac_jump_spot_check", "ac_net_calibrate_guard",
    "ac_slab_plan", "ac_slab_create", "ac_slab_scatter", "ac_slab_gather", "ac_slab_step",
    "ac_slab_set_schedule", "ac_slab_set_graph", "ac_slab_get_part", "ac_slab_launch_count",
    "ac_slab_destroy",
)


class AcGridDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("pitch_x", ctypes.c_int64),
        ("h", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("dt", ctypes.c_double),
    ]


class AcGuard(ctypes.Structure):
    _fields_ = [
        ("steps_per_jump", ctypes.c_int32),
        ("energy_rtol", ctypes.c_double),
        ("max_abs", ctypes.c_double),
        ("residual_tol", ctypes.c_double),
        ("spot_rtol", ctypes.c_double),
        ("spot_samples", ctypes.c_int32),
        ("spot_size", ctypes.c_int32),
        ("spot_seed", ctypes.c_uint64),
    ]


class AcLearnedReport(ctypes.Structure):
    _fields_ = [
        ("jumps", ctypes.c_int64),
        ("fallbacks", ctypes.c_int64),
        ("rejected_nonfinite", ctypes.c_int64),
        ("rejected_energy", ctypes.c_int64),
        ("rejected_max_abs", ctypes.c_int64),
        ("rejected_residual", ctypes.c_int64),
        ("rejected_spot", ctypes.c_int64),
        ("max_residual", ctypes.c_double),
        ("max_spot_rel", ctypes.c_double),
        ("max_spot_abs", ctypes.c_double),
    ]


class AcGuardCalibration(ctypes.Structure):
    _fields_ = [
        ("states", ctypes.c_int32),
        ("plain_residual_max", ctypes.c_double),
        ("net_residual_max", ctypes.c_double),
        ("net_rel_err_median", ctypes.c_double),
        ("net_rel_err_max", ctypes.c_double),
        ("spot_rel_err_max", ctypes.c_double),
    ]


class AcSlabPart(ctypes.Structure):
    _fields_ = [
        ("own_lo", ctypes.c_int64),
        ("own_hi", ctypes.c_int64),
        ("ext_lo", ctypes.c_int64),
        ("ext_hi", ctypes.c_int64),
    ]


def struct_dict(st) -> dict:
    """The fields of a ctypes structure as a plain dict."""
    return {name: getattr(st, name) for name, _ in st._fields_}


class AcTrainConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("eps_cells", ctypes.c_double),
        ("pool", ctypes.c_int32),
        ("trajectory_jumps", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("steps_per_jump", ctypes.c_int32),
        ("lr", ctypes.c_double),
        ("lr_final", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class AcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[ac error {code}] {msg}")
        self.code = code


_lib = None
_build_error = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libac.so (building it first if missing or stale)."""
    global _lib, _build_error
    if _lib is not None:
        return _lib
    if _build_error is not None:  # do not rebuild on every call after a failure
        raise _build_error
    try:
        path = _build.build() if build_if_missing else _build.LIB
    except Exception as e:  # noqa: BLE001 - surfaced to the caller unchanged
        _build_error = e
        raise
    if not os.path.exists(path):
        raise AcError(AC_ERR_UNSUPPORTED, f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    dp = ctypes.POINTER(AcGridDesc)
    sig = {
        "ac_workspace_bytes": [dp, ctypes.POINTER(ctypes.c_size_t)],
        "ac_create": [dp, vp, vp, vp, ctypes.POINTER(vp)],
        "ac_step": [vp, i64],
        "ac_energy": [vp, ctypes.POINTER(dbl)],
        "ac_phase_volume": [vp, ctypes.POINTER(dbl)],
        "ac_observe": [vp, ctypes.POINTER(dbl)],
        "ac_init_sphere": [vp, dbl, dbl, dbl, dbl, dbl, dbl, dbl],
        "ac_init_random": [vp, u64, dbl],
        "ac_init_shape": [vp, i32, dbl, dbl, dbl, dbl, dbl],
        "ac_set_schedule": [vp, i32, i32],
        "ac_get_schedule": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "ac_set_tile": [vp, i32],
        "ac_get_tile": [vp, ctypes.POINTER(i32)],
        "ac_autotune": [vp, i64],
        "ac_set_tune_cache": [ctypes.c_char_p],
        "ac_set_graph": [vp, i32],
        "ac_status": [vp],
        "ac_launch_count": [vp, ctypes.POINTER(i64)],
        "ac_observe_noalloc": [dp, vp, vp, vp],
        "ac_batch_workspace_bytes": [dp, i32, ctypes.POINTER(ctypes.c_size_t)],
        "ac_batch_create": [dp, ctypes.POINTER(vp), i32, vp, vp, ctypes.POINTER(vp)],
        "ac_batch_step": [vp, ctypes.POINTER(i64)],
        "ac_batch_set_schedule": [vp, i32],
        "ac_batch_get_schedule": [vp, ctypes.POINTER(i32)],
        "ac_batch_set_tile": [vp, i32],
        "ac_batch_get_tile": [vp, ctypes.POINTER(i32)],
        "ac_batch_autotune": [vp, i64],
        "ac_batch_set_graph": [vp, i32],
        "ac_batch_observe": [vp, i32, ctypes.POINTER(dbl)],
        "ac_batch_status": [vp],
        "ac_batch_set_wait_limit": [vp, ctypes.c_uint32],
        "ac_batch_launch_count": [vp, ctypes.POINTER(i64)],
        "ac_batch_destroy": [vp],
        "ac_tc_gemm_bf16_n32": [vp, vp, vp, i64, i32, vp],
        "ac_net_param_count": [i32, ctypes.POINTER(i64)],
        "ac_net_create": [i32, vp, ctypes.POINTER(vp)],
        "ac_net_set_params": [vp, vp, i64],
        "ac_net_get_params": [vp, vp, i64],
        "ac_net_forward": [vp, vp, vp, i32, i64, i64, i64, dbl],
        "ac_net_loss_grads": [vp, vp, vp, i32, i64, i64, i64, dbl, ctypes.POINTER(dbl), vp],
        "ac_net_adam": [vp, dbl, dbl, dbl, dbl],
        "ac_net_train_step": [vp, vp, vp, i32, i64, i64, i64, dbl, dbl, ctypes.POINTER(dbl)],
        "ac_net_launch_count": [vp, ctypes.POINTER(i64)],
        "ac_net_destroy": [vp],
        "ac_learned_advance": [vp, vp, i64, ctypes.POINTER(AcGuard), ctypes.POINTER(i64),
                               ctypes.POINTER(AcLearnedReport)],
        "ac_jump_spot_check": [vp, vp, i32, i32, i32, u64, ctypes.POINTER(dbl)],
        "ac_slab_plan": [i64, i32, i32, ctypes.POINTER(AcSlabPart)],
        "ac_slab_create": [dp, i32, i32, vp, ctypes.POINTER(vp)],
        "ac_slab_scatter": [vp, vp],
        "ac_slab_gather": [vp, vp],
        "ac_slab_step": [vp, i64],
        "ac_slab_set_schedule": [vp, i32, i32],
        "ac_slab_set_graph": [vp, i32],
        "ac_slab_get_part": [vp, i32, ctypes.POINTER(AcSlabPart), ctypes.POINTER(i32), ctypes.POINTER(vp)],
        "ac_slab_launch_count": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)],
        "ac_slab_destroy": [vp],
        "ac_net_calibrate_guard": [vp, ctypes.POINTER(AcTrainConfig), dbl, ctypes.POINTER(AcGuard),
                                   ctypes.POINTER(AcGuardCalibration)],
        "ac_net_train": [vp, ctypes.POINTER(AcTrainConfig), vp, ctypes.POINTER(i64)],
        "ac_net_init_params": [vp, u64],
        "ac_jump_residual": [vp, vp, i32, ctypes.POINTER(dbl)],
        "ac_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ac_last_error.argtypes = []
    L.ac_last_error.restype = ctypes.c_char_p
    L.ac_version.argtypes = []
    L.ac_version.restype = ctypes.c_char_p
    _lib = L
    return L


def last_error() -> str:
    return lib().ac_last_error().decode()


def check(rc: int) -> int:
    if rc != AC_OK:
        raise AcError(rc, last_error())
    return rc


# ------------------------------------------------------------ entry points --

def make_desc(ndim: int, dtype: int, nx: int, ny: int, nz: int, pitch_x: int,
              h: float, eps: float, dt: float) -> AcGridDesc:
    return AcGridDesc(ndim, dtype, nx, ny, nz, pitch_x, h, eps, dt)


def ac_workspace_bytes(desc: AcGridDesc) -> int:
    out = ctypes.c_size_t()
    check(lib().ac_workspace_bytes(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def ac_create(desc: AcGridDesc, phi_ptr: int, ws_ptr: int, stream_ptr: int) -> int:
    h = ctypes.c_void_p()
    check(lib().ac_create(ctypes.byref(desc), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(ws_ptr),
                          ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h.value


def ac_step(ctx: int, n: int) -> None:
    check(lib().ac_step(ctypes.c_void_p(ctx), int(n)))


def ac_energy(ctx: int) -> float:
    out = ctypes.c_double()
    check(lib().ac_energy(ctypes.c_void_p(ctx), ctypes.byref(out)))
    return out.value


def ac_phase_volume(ctx: int) -> float:
    out = ctypes.c_double()
    check(lib().ac_phase_volume(ctypes.c_void_p(ctx), ctypes.byref(out)))
    return out.value


def ac_observe(ctx: int, allow_nonfinite: bool = False) -> tuple:
    out = (ctypes.c_double * 3)()
    rc = lib().ac_observe(ctypes.c_void_p(ctx), out)
    if not (allow_nonfinite and rc == AC_ERR_NONFINITE):
        check(rc)
    return out[0], out[1], out[2]


def ac_init_sphere(ctx: int, lower=(0.0, 0.0, 0.0), center=(0.5, 0.5, 0.5), r0: float = 0.25) -> None:
    check(lib().ac_init_sphere(ctypes.c_void_p(ctx), *map(float, lower), *map(float, center), float(r0)))


def ac_init_random(ctx: int, seed: int, amplitude: float = 0.1) -> None:
    check(lib().ac_init_random(ctypes.c_void_p(ctx), int(seed), float(amplitude)))


def ac_init_shape(ctx: int, kind: int, lower=(0.0, 0.0, 0.0), p0: float = 0.0,
                  p1: float = 0.0) -> None:
    check(lib().ac_init_shape(ctypes.c_void_p(ctx), int(kind), float(lower[0]), float(lower[1]),
                              float(lower[2]), float(p0), float(p1)))


def ac_set_schedule(ctx: int, variant: int, k: int) -> None:
    check(lib().ac_set_schedule(ctypes.c_void_p(ctx), int(variant), int(k)))


def ac_get_schedule(ctx: int) -> tuple:
    v, k = ctypes.c_int32(), ctypes.c_int32()
    check(lib().ac_get_schedule(ctypes.c_void_p(ctx), ctypes.byref(v), ctypes.byref(k)))
    return v.value, k.value


def ac_set_tile(ctx: int, tile: int) -> None:
    check(lib().ac_set_tile(ctypes.c_void_p(ctx), int(tile)))


def ac_get_tile(ctx: int) -> int:
    t = ctypes.c_int32()
    check(lib().ac_get_tile(ctypes.c_void_p(ctx), ctypes.byref(t)))
    return t.value


def ac_autotune(ctx: int, steps_per_trial: int = 64) -> None:
    check(lib().ac_autotune(ctypes.c_void_p(ctx), int(steps_per_trial)))


def ac_set_tune_cache(path) -> None:
    """Keep autotuning choices in a text file as well (None: process cache only)."""
    check(lib().ac_set_tune_cache(None if path is None else str(path).encode()))


def ac_set_graph(ctx: int, enable: bool) -> None:
    check(lib().ac_set_graph(ctypes.c_void_p(ctx), int(bool(enable))))


def ac_status(ctx: int) -> int:
    return lib().ac_status(ctypes.c_void_p(ctx))


def ac_launch_count(ctx: int) -> int:
    out = ctypes.c_int64()
    check(lib().ac_launch_count(ctypes.c_void_p(ctx), ctypes.byref(out)))
    return out.value


def ac_observe_noalloc(desc: AcGridDesc, phi_ptr: int, stream_ptr: int, out_ptr: int) -> None:
    """Energy, volume and non-finite count of the field at phi_ptr into the
    three device doubles at out_ptr, without any allocation (see include/ac.h)."""
    check(lib().ac_observe_noalloc(ctypes.byref(desc), ctypes.c_void_p(phi_ptr),
                                   ctypes.c_void_p(stream_ptr), ctypes.c_void_p(out_ptr)))


def ac_destroy(ctx: int) -> None:
    check(lib().ac_destroy(ctypes.c_void_p(ctx)))


def ac_version() -> str:
    return lib().ac_version().decode()


# ------------------------------------------------------------- batched mode --

def _desc_array(descs):
    arr = (AcGridDesc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d
    return arr


def ac_batch_workspace_bytes(descs) -> int:
    out = ctypes.c_size_t()
    check(lib().ac_batch_workspace_bytes(_desc_array(descs), len(descs), ctypes.byref(out)))
    return out.value


def ac_batch_create(descs, phi_ptrs, ws_ptr: int, stream_ptr: int) -> int:
    h = ctypes.c_void_p()
    ptrs = (ctypes.c_void_p * len(phi_ptrs))(*phi_ptrs)
    check(lib().ac_batch_create(_desc_array(descs), ptrs, len(descs), ctypes.c_void_p(ws_ptr),
                                ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h.value


def ac_batch_step(batch: int, n_per_instance) -> None:
    arr = (ctypes.c_int64 * len(n_per_instance))(*[int(n) for n in n_per_instance])
    check(lib().ac_batch_step(ctypes.c_void_p(batch), arr))


def ac_batch_set_schedule(batch: int, k: int) -> None:
    check(lib().ac_batch_set_schedule(ctypes.c_void_p(batch), int(k)))


def ac_batch_set_tile(batch: int, tile: int) -> None:
    check(lib().ac_batch_set_tile(ctypes.c_void_p(batch), int(tile)))


def ac_batch_get_tile(batch: int) -> int:
    t = ctypes.c_int32()
    check(lib().ac_batch_get_tile(ctypes.c_void_p(batch), ctypes.byref(t)))
    return t.value


def ac_batch_get_schedule(batch: int) -> int:
    k = ctypes.c_int32()
    check(lib().ac_batch_get_schedule(ctypes.c_void_p(batch), ctypes.byref(k)))
    return k.value


def ac_batch_autotune(batch: int, steps_per_trial: int = 64) -> None:
    check(lib().ac_batch_autotune(ctypes.c_void_p(batch), int(steps_per_trial)))


def ac_batch_set_graph(batch: int, enable: bool) -> None:
    check(lib().ac_batch_set_graph(ctypes.c_void_p(batch), int(bool(enable))))


def ac_batch_observe(batch: int, i: int, allow_nonfinite: bool = False) -> tuple:
    out = (ctypes.c_double * 3)()
    rc = lib().ac_batch_observe(ctypes.c_void_p(batch), int(i), out)
    if not (allow_nonfinite and rc == AC_ERR_NONFINITE):
        check(rc)
    return out[0], out[1], out[2]


def ac_batch_status(batch: int) -> int:
    return lib().ac_batch_status(ctypes.c_void_p(batch))


def ac_batch_set_wait_limit(batch: int, polls: int) -> None:
    check(lib().ac_batch_set_wait_limit(ctypes.c_void_p(batch), int(polls)))


def ac_batch_launch_count(batch: int) -> int:
    out = ctypes.c_int64()
    check(lib().ac_batch_launch_count(ctypes.c_void_p(batch), ctypes.byref(out)))
    return out.value


def ac_batch_destroy(batch: int) -> None:
    check(lib().ac_batch_destroy(ctypes.c_void_p(batch)))


def ac_tc_gemm_bf16_n32(a_ptr: int, b_ptr: int, d_ptr: int, m: int, k: int, stream_ptr: int) -> None:
    check(lib().ac_tc_gemm_bf16_n32(ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr),
                                    ctypes.c_void_p(d_ptr), int(m), int(k), ctypes.c_void_p(stream_ptr)))


# ---------------------------------------------------------- learned stepper --

def ac_net_param_count(ndim: int) -> int:
    out = ctypes.c_int64()
    check(lib().ac_net_param_count(int(ndim), ctypes.byref(out)))
    return out.value


def ac_net_create(ndim: int, stream_ptr: int) -> int:
    h = ctypes.c_void_p()
    check(lib().ac_net_create(int(ndim), ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    return h.value


def ac_net_set_params(net: int, params_f32) -> None:
    import numpy as np
    a = np.ascontiguousarray(params_f32, dtype=np.float32)
    check(lib().ac_net_set_params(ctypes.c_void_p(net), a.ctypes.data_as(ctypes.c_void_p), a.size))


def ac_net_get_params(net: int, count: int):
    import numpy as np
    a = np.empty(count, dtype=np.float32)
    check(lib().ac_net_get_params(ctypes.c_void_p(net), a.ctypes.data_as(ctypes.c_void_p), count))
    return a


def ac_net_forward(net: int, phi_ptr: int, out_ptr: int, batch: int, nx: int, ny: int, nz: int,
                   scale: float) -> None:
    check(lib().ac_net_forward(ctypes.c_void_p(net), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(out_ptr),
                               int(batch), int(nx), int(ny), int(nz), float(scale)))


def ac_net_loss_grads(net: int, phi_ptr: int, target_ptr: int, batch: int, nx: int, ny: int, nz: int,
                      scale: float, want_grads: bool = False):
    import numpy as np
    loss = ctypes.c_double()
    grads = None
    gp = None
    if want_grads:
        cnt = ctypes.c_int64()
        # parameter count of this network's dimension: nz > 1 means 3D
        check(lib().ac_net_param_count(3 if nz > 1 else 2, ctypes.byref(cnt)))
        grads = np.empty(cnt.value, dtype=np.float32)
        gp = grads.ctypes.data_as(ctypes.c_void_p)
    check(lib().ac_net_loss_grads(ctypes.c_void_p(net), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(target_ptr),
                                  int(batch), int(nx), int(ny), int(nz), float(scale), ctypes.byref(loss), gp))
    return loss.value, grads


def ac_net_adam(net: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    check(lib().ac_net_adam(ctypes.c_void_p(net), float(lr), float(beta1), float(beta2), float(eps)))


def ac_net_train_step(net: int, phi_ptr: int, target_ptr: int, batch: int, nx: int, ny: int, nz: int,
                      scale: float, lr: float) -> float:
    loss = ctypes.c_double()
    check(lib().ac_net_train_step(ctypes.c_void_p(net), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(target_ptr),
                                  int(batch), int(nx), int(ny), int(nz), float(scale), float(lr),
                                  ctypes.byref(loss)))
    return loss.value


def ac_net_launch_count(net: int) -> int:
    out = ctypes.c_int64()
    check(lib().ac_net_launch_count(ctypes.c_void_p(net), ctypes.byref(out)))
    return out.value


def ac_net_destroy(net: int) -> None:
    check(lib().ac_net_destroy(ctypes.c_void_p(net)))


def ac_learned_advance(ctx: int, net: int, jumps: int, guard: "AcGuard", with_report: bool = False):
    """Returns the number of rejected jumps, or (that number, the report as
    a dict) with with_report=True."""
    fb = ctypes.c_int64()
    rep = AcLearnedReport()
    check(lib().ac_learned_advance(ctypes.c_void_p(ctx), ctypes.c_void_p(net), int(jumps),
                                   ctypes.byref(guard), ctypes.byref(fb), ctypes.byref(rep)))
    return (fb.value, struct_dict(rep)) if with_report else fb.value


def ac_jump_spot_check(ctx: int, phat_ptr: int, steps: int, samples: int = 0, size: int = 0,
                       seed: int = 0) -> tuple:
    """(max |phat - ref|, relative L2 error, cells checked) of the spot check."""
    out = (ctypes.c_double * 3)()
    check(lib().ac_jump_spot_check(ctypes.c_void_p(ctx), ctypes.c_void_p(phat_ptr), int(steps),
                                   int(samples), int(size), int(seed), out))
    return out[0], out[1], out[2]


def ac_net_calibrate_guard(net: int, cfg: "AcTrainConfig", residual_factor: float, guard: "AcGuard") -> dict:
    """Sets guard.residual_tol in place; returns the calibration report."""
    rep = AcGuardCalibration()
    check(lib().ac_net_calibrate_guard(ctypes.c_void_p(net), ctypes.byref(cfg), float(residual_factor),
                                       ctypes.byref(guard), ctypes.byref(rep)))
    return struct_dict(rep)


def ac_net_train(net: int, cfg: "AcTrainConfig"):
    """Returns (loss history as a numpy array, trajectories used)."""
    import numpy as np
    hist = np.zeros(cfg.iterations, dtype=np.float64)
    used = ctypes.c_int64()
    check(lib().ac_net_train(ctypes.c_void_p(net), ctypes.byref(cfg), hist.ctypes.data_as(ctypes.c_void_p),
                             ctypes.byref(used)))
    return hist, used.value


def ac_net_init_params(net: int, seed: int) -> None:
    check(lib().ac_net_init_params(ctypes.c_void_p(net), int(seed)))


def ac_jump_residual(ctx: int, phat_ptr: int, steps: int) -> tuple:
    out = (ctypes.c_double * 2)()
    check(lib().ac_jump_residual(ctypes.c_void_p(ctx), ctypes.c_void_p(phat_ptr), int(steps), out))
    return out[0], out[1]


def ac_slab_plan(extent: int, parts: int, halo: int) -> list:
    """[(own_lo, own_hi, ext_lo, ext_hi)] per part (host arithmetic only)."""
    out = (AcSlabPart * max(1, int(parts)))()
    check(lib().ac_slab_plan(int(extent), int(parts), int(halo), out))
    return [(p.own_lo, p.own_hi, p.ext_lo, p.ext_hi) for p in out[:int(parts)]]


def ac_slab_create(desc: "AcGridDesc", parts: int, halo: int, stream: int) -> int:
    out = ctypes.c_void_p()
    check(lib().ac_slab_create(ctypes.byref(desc), int(parts), int(halo), ctypes.c_void_p(stream),
                               ctypes.byref(out)))
    return out.value


def ac_slab_scatter(slab: int, phi_ptr: int) -> None:
    check(lib().ac_slab_scatter(ctypes.c_void_p(slab), ctypes.c_void_p(phi_ptr)))


def ac_slab_gather(slab: int, phi_ptr: int) -> None:
    check(lib().ac_slab_gather(ctypes.c_void_p(slab), ctypes.c_void_p(phi_ptr)))


def ac_slab_step(slab: int, n: int) -> None:
    check(lib().ac_slab_step(ctypes.c_void_p(slab), int(n)))


def ac_slab_set_schedule(slab: int, variant: int, k: int) -> None:
    check(lib().ac_slab_set_schedule(ctypes.c_void_p(slab), int(variant), int(k)))


def ac_slab_set_graph(slab: int, enable: bool) -> None:
    check(lib().ac_slab_set_graph(ctypes.c_void_p(slab), int(bool(enable))))


def ac_slab_get_part(slab: int, part: int) -> tuple:
    """((own_lo, own_hi, ext_lo, ext_hi), halo, device pointer of the part's field)."""
    pl = AcSlabPart()
    halo = ctypes.c_int32()
    ptr = ctypes.c_void_p()
    check(lib().ac_slab_get_part(ctypes.c_void_p(slab), int(part), ctypes.byref(pl), ctypes.byref(halo),
                                 ctypes.byref(ptr)))
    return (pl.own_lo, pl.own_hi, pl.ext_lo, pl.ext_hi), halo.value, ptr.value


def ac_slab_launch_count(slab: int) -> tuple:
    k, c = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ac_slab_launch_count(ctypes.c_void_p(slab), ctypes.byref(k), ctypes.byref(c)))
    return k.value, c.value


def ac_slab_destroy(slab: int) -> None:
    check(lib().ac_slab_destroy(ctypes.c_void_p(slab)))
