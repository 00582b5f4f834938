"""Slab decomposition of one grid along its slowest axis (z in 3D, y in 2D).

A step of a cell reads only its neighbours, so ``b`` steps of a slab's own
planes need the ``b`` planes beyond each face it shares with another slab.
Each part therefore holds ``halo`` extra planes on such faces, advances its
extended slab by at most ``halo`` steps with the ordinary stepper (the
zero-Neumann clamp at the artificial face of an extended slab corrupts only
its halo planes, one plane per step) and then refreshes its halos from the
neighbours' owned planes.  The owned planes are bit for bit those of the
undivided grid (FP16 storage rounds once per pass: bit for bit only where
the passes end at the same steps).  The plan comes from ``ac_slab_plan`` in
the C library.

``Slab``: all parts in this process on one device (``ac_slab_*``).
``DistributedSlab``: one part per rank of a ``torch.distributed`` group;
the halo exchange is a batch of point-to-point sends and receives of
contiguous plane blocks between neighbouring ranks.  The field of a part is
any tensor whose first axis holds its planes [ext_lo, ext_hi); the stepping
is a callable, normally ``Simulation.step`` on that extended slab (see
``DistributedSlab.on_device``).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


def plan(extent: int, parts: int, halo: int) -> list:
    """[(own_lo, own_hi, ext_lo, ext_hi)] of every part."""
    return L.ac_slab_plan(extent, parts, halo)


class Slab:
    """All parts of a decomposed grid in this process (``ac_slab_*``).

    ``shape`` is (ny, nx) or (nz, ny, nx); fields move in and out of the
    parts as whole-grid tensors of the ``Simulation`` layout.
    """

    def __init__(self, shape, h, eps, dt, parts: int, halo: int = 0, dtype="f32", device="cuda",
                 stream: torch.cuda.Stream | None = None, pitch_x: int | None = None):
        from .sim import Simulation
        # a full-size Simulation holds the whole field (scatter source, gather target)
        self.full = Simulation(shape, h, eps, dt, dtype=dtype, device=device, stream=stream, pitch_x=pitch_x)
        self.stream = self.full.stream
        self.handle = L.ac_slab_create(self.full.desc, parts, halo, self.stream.cuda_stream)
        self.parts = parts
        _, self.halo, _ = L.ac_slab_get_part(self.handle, 0)

    def load(self, array) -> None:
        self.full.load(array)
        L.ac_slab_scatter(self.handle, self.full._buf.data_ptr())

    def scatter(self) -> None:
        L.ac_slab_scatter(self.handle, self.full._buf.data_ptr())

    def gather(self) -> None:
        L.ac_slab_gather(self.handle, self.full._buf.data_ptr())

    def step(self, n: int) -> None:
        L.ac_slab_step(self.handle, n)

    def set_schedule(self, variant: int, k: int) -> None:
        L.ac_slab_set_schedule(self.handle, variant, k)

    def set_graph(self, enable: bool) -> None:
        L.ac_slab_set_graph(self.handle, enable)

    def part(self, i: int) -> tuple:
        return L.ac_slab_get_part(self.handle, i)

    def launch_count(self) -> tuple:
        return L.ac_slab_launch_count(self.handle)

    def to_numpy(self) -> np.ndarray:
        self.gather()
        return self.full.to_numpy()

    def close(self) -> None:
        if getattr(self, "handle", None):
            L.ac_slab_destroy(self.handle)
            self.handle = None
        if getattr(self, "full", None) is not None:
            self.full.close()
            self.full = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DistributedSlab:
    """This rank's part of a grid split over the ranks of ``group``.

    ``field``: tensor whose first axis holds planes [ext_lo, ext_hi) of the
    rank's plan entry (the halos included); ``step_fn(n)`` advances that
    extended slab by n steps in place.  ``step(n)`` runs blocks of at most
    ``halo`` steps with a halo exchange before every block but the first
    after ``mark_fresh()`` (call it once the halos hold current values, e.g.
    right after loading the field).
    """

    def __init__(self, extent: int, halo: int, field: torch.Tensor, step_fn, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.halo = int(halo)
        self.plan = plan(extent, self.world, self.halo)
        self.own_lo, self.own_hi, self.ext_lo, self.ext_hi = self.plan[self.rank]
        if field.shape[0] != self.ext_hi - self.ext_lo:
            raise ValueError(f"field holds {field.shape[0]} planes, the plan {self.ext_hi - self.ext_lo}")
        self.field = field
        self.step_fn = step_fn
        self.stream = None  # the CUDA stream step_fn runs on (None: the current stream)
        self.fresh = False
        self.exchanges = 0

    @classmethod
    def on_device(cls, shape, h, eps, dt, halo: int, dtype="f32", device="cuda", group=None,
                  stream: torch.cuda.Stream | None = None):
        """A part backed by a Simulation over this rank's extended slab.
        Returns (DistributedSlab, Simulation)."""
        import torch.distributed as dist
        from .sim import Simulation
        shape = tuple(int(s) for s in shape)
        p = plan(shape[0], dist.get_world_size(group), halo)[dist.get_rank(group)]
        local = (p[3] - p[2],) + shape[1:]
        sim = Simulation(local, h, eps, dt, dtype=dtype, device=device, stream=stream)
        field = sim.padded if len(shape) == 3 else sim.padded[0]
        ds = cls(shape[0], halo, field, sim.step, group=group)
        ds.stream = sim.stream
        return ds, sim

    def owned(self) -> torch.Tensor:
        """View of the planes this rank owns."""
        return self.field[self.own_lo - self.ext_lo:self.own_hi - self.ext_lo]

    def mark_fresh(self) -> None:
        self.fresh = True

    def exchange(self) -> None:
        """Refresh both halos from the neighbouring ranks' owned planes."""
        dist = self.dist
        f, lo = self.field, self.ext_lo
        # device fields: the transfers run in the order of the current stream,
        # so it waits for the steps first and the steps wait for the transfers
        cur = None
        if f.is_cuda and self.stream is not None:
            cur = torch.cuda.current_stream(f.device)
            cur.wait_stream(self.stream)
        ops = []
        if self.rank > 0:
            n_lo = self.own_lo - self.ext_lo  # my lower halo <- last planes of rank - 1
            peer = dist.get_global_rank(self.group, self.rank - 1) if self.group else self.rank - 1
            ops.append(dist.P2POp(dist.irecv, f[0:n_lo], peer, self.group))
            # rank - 1's upper halo <- my first planes
            _, _, _, prev_ext_hi = self.plan[self.rank - 1]
            n_up = prev_ext_hi - self.own_lo
            ops.append(dist.P2POp(dist.isend, f[self.own_lo - lo:self.own_lo - lo + n_up].contiguous(), peer,
                                  self.group))
        if self.rank + 1 < self.world:
            # my upper halo <- first planes of rank + 1
            peer = dist.get_global_rank(self.group, self.rank + 1) if self.group else self.rank + 1
            ops.append(dist.P2POp(dist.irecv, f[self.own_hi - lo:self.ext_hi - lo], peer, self.group))
            # rank + 1's lower halo <- my last planes
            nxt_ext_lo = self.plan[self.rank + 1][2]
            ops.append(dist.P2POp(dist.isend, f[nxt_ext_lo - lo:self.own_hi - lo].contiguous(), peer,
                                  self.group))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
            self.exchanges += 1
        if cur is not None:
            self.stream.wait_stream(cur)
        self.fresh = True

    def step(self, n: int) -> None:
        n = int(n)
        while n > 0:
            b = min(n, self.halo)
            if not self.fresh:
                self.exchange()
            self.step_fn(b)
            if self.world > 1:
                self.fresh = False
            n -= b
