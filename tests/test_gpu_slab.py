"""Slab decomposition on the GPU: several parts of one grid on one device,
each stepped by the library's own kernels on its extended slab, halos
refreshed by device copies between blocks.  The owned planes must equal
the undivided grid's steps bit for bit (same kernels, same inputs per
cell), and so match the FP64 oracle within the usual tolerances."""
import numpy as np
import pytest

import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl
from paper_2105_09671_gb300.slab import Slab

from gpu_util import assert_parity, oracle_run

pytestmark = pytest.mark.gpu


def _field(shape, seed):
    return wl.smooth_field(shape, seed=seed) + 0.05 * np.random.default_rng(seed).uniform(-1, 1, shape)


@pytest.mark.parametrize("shape,parts,halo,n,dtype", [
    ((96, 70), 2, 8, 37, "f32"),           # 2D split in y, remainder block
    ((130, 64), 3, 0, 50, "f32"),          # 2D, default halo (8), uneven parts
    ((40, 24, 36), 2, 4, 21, "f32"),       # 3D split in z
    ((53, 20, 17), 4, 0, 30, "f32"),       # 3D, four uneven parts, ragged x
    ((33, 16, 16), 3, 2, 11, "f64"),       # FP64: the direct kernel, one step per launch
    ((64, 64), 2, 6, 25, "f16s"),          # FP16 storage
])
def test_slabs_equal_the_undivided_grid(shape, parts, halo, n, dtype):
    h = 1.0 / max(shape)
    eps, dt = 3.0 * h, 0.1 * h * h
    phi0 = _field(shape, seed=sum(shape))
    whole = ac.Simulation(shape, h, eps, dt, dtype=dtype)
    slab = Slab(shape, h, eps, dt, parts=parts, halo=halo, dtype=dtype)
    try:
        whole.load(phi0)
        whole.step(n)
        ref = whole.to_numpy()
        slab.load(phi0)
        slab.step(n)
        got = slab.to_numpy()
        if dtype == "f16s":
            # FP16 storage rounds at the end of each pass; the slab's blocks
            # of `halo` steps put pass boundaries elsewhere than the whole
            # grid's plan, so the two agree to the storage rounding only
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= 4e-3
        else:
            assert np.array_equal(got, ref)
        assert_parity(got.astype(np.float64), oracle_run(phi0, h, eps, dt, n, dtype), dtype, "slab")
        kernels, copies = slab.launch_count()
        blocks = -(-n // slab.halo)
        assert copies == 2 * parts + 2 * (parts - 1) * (blocks - 1)  # scatter, exchanges, gather
        assert kernels > 0
    finally:
        slab.close()
        whole.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_slabs_on_every_3d_depth(k):
    shape = (48, 40, 64)
    h = 1.0 / 64
    eps, dt = 3.0 * h, 0.1 * h * h
    phi0 = _field(shape, seed=k)
    whole = ac.Simulation(shape, h, eps, dt, dtype="f32")
    slab = Slab(shape, h, eps, dt, parts=3, halo=2 * k, dtype="f32")
    try:
        whole.set_schedule(ac.AC_VARIANT_STREAM, k)
        slab.set_schedule(ac.AC_VARIANT_STREAM, k)
        whole.load(phi0)
        whole.step(6 * k + 1)
        slab.load(phi0)
        slab.step(6 * k + 1)
        assert np.array_equal(slab.to_numpy(), whole.to_numpy())
    finally:
        slab.close()
        whole.close()


def test_sphere_512_in_two_slabs_matches_the_whole_grid():
    # the benchmark grid, 200 steps, split in two along z
    w = wl.SPHERE_512
    whole = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype="f32")
    slab = Slab(w.shape, w.h, w.eps, w.dt, parts=2, dtype="f32")
    try:
        whole.init_sphere(r0=w.r0)
        slab.full.init_sphere(r0=w.r0)
        slab.scatter()
        whole.step(200)
        slab.step(200)
        slab.gather()
        import torch
        torch.cuda.synchronize()
        assert torch.equal(slab.full.phi, whole.phi)
    finally:
        slab.close()
        whole.close()


def test_distributed_slab_on_device_single_rank():
    # the one-rank-per-part layer on a device: with one rank there is nothing
    # to exchange, and the part is the whole grid stepped by its Simulation
    import os
    import socket
    import torch
    import torch.distributed as dist
    from paper_2105_09671_gb300.slab import DistributedSlab
    if dist.is_initialized():
        pytest.skip("a process group already exists")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        shape = (24, 20, 36)
        h = 1.0 / 36
        eps, dt = 3.0 * h, 0.1 * h * h
        phi0 = _field(shape, seed=4)
        ds, sim = DistributedSlab.on_device(shape, h, eps, dt, halo=4, dtype="f32")
        whole = ac.Simulation(shape, h, eps, dt, dtype="f32")
        try:
            assert (ds.own_lo, ds.own_hi, ds.ext_lo, ds.ext_hi) == (0, 24, 0, 24)
            sim.load(phi0)
            ds.mark_fresh()
            ds.step(10)
            whole.load(phi0)
            whole.step(10)
            assert ds.exchanges == 0
            torch.cuda.synchronize()
            assert np.array_equal(sim.to_numpy(), whole.to_numpy())
            assert torch.equal(ds.owned()[:, :, :36].cpu(), torch.from_numpy(sim.to_numpy()))
        finally:
            whole.close()
            sim.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,parts,n", [((40, 24, 36), 3, 13), ((96, 70), 2, 37)])
def test_slab_graph_replay_equals_direct_launches(shape, parts, n):
    # the captured sequence (every part's launches and the halo copies) is
    # replayed for repeated step counts and re-captured when the count or
    # the halo state at the start changes
    import torch
    h = 1.0 / max(shape)
    eps, dt = 3.0 * h, 0.1 * h * h
    phi0 = _field(shape, seed=7)
    stream = torch.cuda.Stream()
    direct = Slab(shape, h, eps, dt, parts=parts, halo=4, dtype="f32", stream=stream)
    graph = Slab(shape, h, eps, dt, parts=parts, halo=4, dtype="f32", stream=stream)
    try:
        graph.set_graph(True)
        for sl in (direct, graph):
            sl.load(phi0)
            sl.step(n)       # halos fresh after the load
            sl.step(n)       # stale halos: a second capture
            sl.step(n)       # replay of the second
            sl.step(n + 2)   # another count
        assert np.array_equal(graph.to_numpy(), direct.to_numpy())
        assert graph.launch_count() == direct.launch_count()
    finally:
        direct.close()
        graph.close()


def test_slab_graph_needs_a_stream():
    shape = (32, 32)
    slab = Slab(shape, 1 / 32, 3 / 32, 0.1 / 32 ** 2, parts=2, dtype="f32")
    try:
        with pytest.raises(RuntimeError):
            slab.set_graph(True)
    finally:
        slab.close()
