"""PyTorch-facing handle for one Allen-Cahn grid.

PyTorch provides the device memory (the field and its ping-pong workspace)
and the CUDA stream; every step, reduction and initial condition runs in
``libac.so`` through the C ABI.  Nothing here computes any part of the method.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

_TORCH = {L.AC_F64: torch.float64, L.AC_F32: torch.float32, L.AC_F16S: torch.float16}
_NUMPY = {L.AC_F64: np.float64, L.AC_F32: np.float32, L.AC_F16S: np.float16}
DTYPES = {"f64": L.AC_F64, "f32": L.AC_F32, "f16s": L.AC_F16S}


def _dtype_code(dtype) -> int:
    if isinstance(dtype, str):
        return DTYPES[dtype]
    return int(dtype)


class Simulation:
    """A grid of shape (ny, nx) or (nz, ny, nx) resident on a CUDA device.

    ``pitch_x`` defaults to nx rounded up to 128 bytes.  ``stream`` is a
    ``torch.cuda.Stream`` (default: the current stream); all library work is
    ordered on it.
    """

    def __init__(self, shape, h: float, eps: float, dt: float, dtype="f32", device="cuda",
                 stream: torch.cuda.Stream | None = None, pitch_x: int | None = None):
        if not torch.cuda.is_available():
            raise L.AcError(L.AC_ERR_UNSUPPORTED, "a CUDA device is required")
        self.code = _dtype_code(dtype)
        shape = tuple(int(s) for s in shape)
        if len(shape) == 2:
            self.nz, self.ny, self.nx = 1, shape[0], shape[1]
            self.ndim = 2
        elif len(shape) == 3:
            self.nz, self.ny, self.nx = shape
            self.ndim = 3
        else:
            raise ValueError("shape must have 2 or 3 entries")
        self.shape = shape
        es = np.dtype(_NUMPY[self.code]).itemsize
        per = 128 // es
        self.pitch_x = int(pitch_x) if pitch_x is not None else -(-self.nx // per) * per
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h, self.eps, self.dt = float(h), float(eps), float(dt)
        self.desc = L.make_desc(self.ndim, self.code, self.nx, self.ny, self.nz, self.pitch_x,
                                self.h, self.eps, self.dt)
        nbytes = L.ac_workspace_bytes(self.desc)
        n = nbytes // es
        tdt = _TORCH[self.code]
        with torch.cuda.device(self.device):
            self._buf = torch.zeros(n, dtype=tdt, device=self.device)
            self._ws = torch.zeros(n, dtype=tdt, device=self.device)
            self.ctx = L.ac_create(self.desc, self._buf.data_ptr(), self._ws.data_ptr(),
                                   self.stream.cuda_stream)

    # -- field access (views of the caller-owned buffer) ---------------------
    @property
    def phi(self) -> torch.Tensor:
        """The field as a strided view, shape ``self.shape``."""
        v = self._buf.view(self.nz, self.ny, self.pitch_x)[:, :, : self.nx]
        return v[0] if self.ndim == 2 else v

    @property
    def padded(self) -> torch.Tensor:
        return self._buf.view(self.nz, self.ny, self.pitch_x)

    def load(self, array) -> None:
        """Copy a host array (any float dtype) into the field, rounding to the storage type."""
        a = np.asarray(array)
        if a.shape != self.shape:
            raise ValueError(f"shape {a.shape} != {self.shape}")
        t = torch.from_numpy(np.ascontiguousarray(a.astype(_NUMPY[self.code])))
        with torch.cuda.stream(self.stream):
            self.phi.copy_(t.to(self.device, non_blocking=False))

    def to_numpy(self) -> np.ndarray:
        self.stream.synchronize()
        return self.phi.cpu().numpy().copy()

    # -- the C ABI -------------------------------------------------------------
    def step(self, n: int) -> None:
        L.ac_step(self.ctx, n)

    def energy(self) -> float:
        return L.ac_energy(self.ctx)

    def phase_volume(self) -> float:
        return L.ac_phase_volume(self.ctx)

    def observe(self, allow_nonfinite: bool = False):
        return L.ac_observe(self.ctx, allow_nonfinite)

    def init_sphere(self, r0: float = 0.25, center=(0.5, 0.5, 0.5), lower=(0.0, 0.0, 0.0)) -> None:
        L.ac_init_sphere(self.ctx, lower, center, r0)

    def init_random(self, seed: int, amplitude: float = 0.1) -> None:
        L.ac_init_random(self.ctx, seed, amplitude)

    def init_shape(self, kind: str, lower=(0.0, 0.0, 0.0), **params) -> None:
        """Dumbbell (r0), star, or torus (r1, r2) of Section 3.1 on the device."""
        if kind == "dumbbell":
            L.ac_init_shape(self.ctx, L.AC_SHAPE_DUMBBELL, lower, params.get("r0", 0.2))
        elif kind == "star":
            L.ac_init_shape(self.ctx, L.AC_SHAPE_STAR, lower)
        elif kind == "torus":
            L.ac_init_shape(self.ctx, L.AC_SHAPE_TORUS, lower, params.get("r1", 0.4),
                            params.get("r2", 0.3))
        else:
            raise ValueError(f"unknown shape {kind!r}")

    def set_schedule(self, variant: int, k: int) -> None:
        L.ac_set_schedule(self.ctx, variant, k)

    def schedule(self):
        return L.ac_get_schedule(self.ctx)

    def set_tile(self, tile: int) -> None:
        """3D streaming tile shape (0..AC_NUM_TILES_3D-1, or -1 for auto)."""
        L.ac_set_tile(self.ctx, tile)

    def tile(self) -> int:
        return L.ac_get_tile(self.ctx)

    def autotune(self, steps_per_trial: int = 64) -> None:
        L.ac_autotune(self.ctx, steps_per_trial)

    def set_graph(self, enable: bool) -> None:
        L.ac_set_graph(self.ctx, enable)

    def launch_count(self) -> int:
        return L.ac_launch_count(self.ctx)

    def status(self) -> int:
        return L.ac_status(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            L.ac_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent 2D grids stepped by one persistent kernel launch.

    ``specs`` is a list of (shape, h, eps, dt); every grid gets its own field
    (a PyTorch tensor) and a slice of one shared workspace.  All grids share
    one storage type and the stream.
    """

    def __init__(self, specs, dtype="f32", device="cuda", stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise L.AcError(L.AC_ERR_UNSUPPORTED, "a CUDA device is required")
        self.code = _dtype_code(dtype)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        es = np.dtype(_NUMPY[self.code]).itemsize
        per = 128 // es
        self.shapes, self.descs, self.fields = [], [], []
        tdt = _TORCH[self.code]
        for shape, h, eps, dt in specs:
            ny, nx = (int(shape[0]), int(shape[1]))
            pitch = -(-nx // per) * per
            self.shapes.append((ny, nx))
            self.descs.append(L.make_desc(2, self.code, nx, ny, 1, pitch, float(h), float(eps), float(dt)))
            self.fields.append(torch.zeros(ny * pitch, dtype=tdt, device=self.device))
        nbytes = L.ac_batch_workspace_bytes(self.descs)
        self._ws = torch.zeros(nbytes // es + 256 // es, dtype=tdt, device=self.device)
        ws_ptr = self._ws.data_ptr()
        ws_ptr = -(-ws_ptr // 256) * 256
        self.handle = L.ac_batch_create(self.descs, [f.data_ptr() for f in self.fields], ws_ptr,
                                        self.stream.cuda_stream)

    def __len__(self):
        return len(self.fields)

    def phi(self, i: int) -> torch.Tensor:
        ny, nx = self.shapes[i]
        return self.fields[i].view(ny, -1)[:, :nx]

    def load(self, i: int, array) -> None:
        a = np.asarray(array)
        t = torch.from_numpy(np.ascontiguousarray(a.astype(_NUMPY[self.code])))
        with torch.cuda.stream(self.stream):
            self.phi(i).copy_(t.to(self.device))

    def to_numpy(self, i: int) -> np.ndarray:
        self.stream.synchronize()
        return self.phi(i).cpu().numpy().copy()

    def step(self, n_per_instance) -> None:
        if np.isscalar(n_per_instance):
            n_per_instance = [int(n_per_instance)] * len(self)
        L.ac_batch_step(self.handle, n_per_instance)

    def set_schedule(self, k: int) -> None:
        L.ac_batch_set_schedule(self.handle, k)

    def schedule(self) -> int:
        return L.ac_batch_get_schedule(self.handle)

    def set_tile(self, tile: int) -> None:
        L.ac_batch_set_tile(self.handle, tile)

    def tile(self) -> int:
        return L.ac_batch_get_tile(self.handle)

    def autotune(self, steps_per_trial: int = 64) -> None:
        L.ac_batch_autotune(self.handle, steps_per_trial)

    def set_graph(self, enable: bool) -> None:
        L.ac_batch_set_graph(self.handle, enable)

    def observe(self, i: int):
        return L.ac_batch_observe(self.handle, i)

    def status(self) -> int:
        return L.ac_batch_status(self.handle)

    def set_wait_limit(self, polls: int) -> None:
        L.ac_batch_set_wait_limit(self.handle, polls)

    def launch_count(self) -> int:
        return L.ac_batch_launch_count(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            L.ac_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
