"""Parity of the CUDA stepper with the FP64 oracle, element by element.

Every schedule the library offers (the direct kernel and each streaming
depth k) is run on the same stored inputs as the oracle.  Sizes span several
tiles with ragged tails; degenerate grids (single cells, single rows /
columns / planes) and padded pitches are included.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import assert_parity, gpu_run, oracle_run, rel_l2, schedules, stored

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(shape):
    h = 1.0 / max(shape)
    return h, 2.5 * h, 0.1 * h * h


# ------------------------------------------------ the 64^2 circle workload --

@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_circle64_1000_steps_every_schedule(dtype):
    w = wl.CIRCLE_64
    phi0 = oracle.init_sphere(w.shape, w.h, w.r0, w.eps)
    ref = oracle_run(phi0, w.h, w.eps, w.dt, w.steps, dtype)
    for variant, k, tile in schedules(2, dtype):
        out = gpu_run(phi0, w.h, w.eps, w.dt, w.steps, dtype, variant, k, tile)
        assert_parity(out, ref, dtype, f"{dtype} variant {variant} k {k} tile {tile}")


def test_default_schedule_and_graph_replay_match():
    w = wl.CIRCLE_64
    phi0 = oracle.init_sphere(w.shape, w.h, w.r0, w.eps)
    ref = oracle_run(phi0, w.h, w.eps, w.dt, 300, "f32")
    import torch
    s = torch.cuda.Stream()
    sim = ac.Simulation(w.shape, w.h, w.eps, w.dt, dtype="f32", stream=s)
    try:
        sim.load(phi0)
        sim.set_graph(True)
        for _ in range(3):
            sim.step(100)      # captured once, replayed twice
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    assert_parity(out, ref, "f32", "graph replay")


# ------------------------------------------------- ragged and degenerate ---

SHAPES_2D = [(1, 1), (1, 37), (29, 1), (3, 5), (33, 97), (130, 129), (250, 300)]
SHAPES_3D = [(1, 1, 1), (2, 3, 5), (9, 17, 33), (5, 40, 150), (33, 36, 131)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_ragged_shapes_every_schedule(shape, dtype):
    h, eps, dt = _params(shape)
    phi0 = wl.smooth_field(shape, seed=sum(shape)) + 0.05 * wl.random_field(shape, seed=7)
    for variant, k, tile in schedules(len(shape), dtype):
        for n in (1, k + 2, 2 * k + 1):
            ref = oracle_run(phi0, h, eps, dt, n, dtype)
            out = gpu_run(phi0, h, eps, dt, n, dtype, variant, k, tile)
            assert_parity(out, ref, dtype, f"{shape} {dtype} v{variant} k{k} t{tile} n{n}")


def test_3d_plane_counts_cover_every_unrolled_remainder():
    """nz = 1..13 on a one-tile xy grid: the plane loop (unrolled by 3 or 6)
    ends on every remainder, items have fewer planes than TMA stages, and
    from nz = 8 on the grid splits into several z-chunks."""
    from paper_2105_09671_gb300 import _lib as L
    for nz in range(1, 14):
        shape = (nz, 20, 24)
        h, eps, dt = _params(shape)
        phi0 = wl.smooth_field(shape, seed=nz) + 0.05 * wl.random_field(shape, seed=nz + 1)
        for variant, k, tile in schedules(3, "f32"):
            if variant != L.AC_VARIANT_STREAM:
                continue
            n = 2 * k + 1
            ref = oracle_run(phi0, h, eps, dt, n, "f32")
            out = gpu_run(phi0, h, eps, dt, n, "f32", variant, k, tile)
            assert_parity(out, ref, "f32", f"nz {nz} k{k} t{tile}")


@pytest.mark.parametrize("shape", [(37, 45), (7, 19, 23)])
def test_f16_storage_ragged(shape):
    h, eps, dt = _params(shape)
    phi0 = wl.smooth_field(shape, seed=3)
    ref = oracle_run(phi0, h, eps, dt, 40, "f16s")
    for variant, k, tile in schedules(len(shape), "f16s"):
        out = gpu_run(phi0, h, eps, dt, 40, "f16s", variant, k, tile)
        assert_parity(out, ref, "f16s", f"{shape} v{variant} k{k}")


@pytest.mark.parametrize("shape,dtype", [((20, 27), "f32"), ((6, 11, 13), "f64"), ((9, 50), "f16s")])
def test_padding_never_read_or_written(shape, dtype):
    import torch
    h, eps, dt = _params(shape)
    phi0 = wl.smooth_field(shape, seed=1)
    nx = shape[-1]
    es = {"f64": 8, "f32": 4, "f16s": 2}[dtype]
    pitch = -(-(nx + 19) // (16 // es)) * (16 // es)
    for variant, k, tile in schedules(len(shape), dtype):
        sim = ac.Simulation(shape, h, eps, dt, dtype=dtype, pitch_x=pitch)
        try:
            sim.set_schedule(variant, k)
            sim.set_tile(tile)
            sim.padded.fill_(float("nan"))
            sim._ws.fill_(float("nan"))
            sim.load(phi0)
            sim.step(2 * k + 1)
            torch.cuda.synchronize()
            pad = sim.padded[:, :, nx:]
            assert torch.isnan(pad).all(), "padding written"
            out = sim.to_numpy().astype(np.float64)
        finally:
            sim.close()
        ref = oracle_run(phi0, h, eps, dt, 2 * k + 1, dtype)
        assert np.isfinite(out).all(), "padding leaked into the field"
        assert_parity(out, ref, dtype, f"padded v{variant} k{k} t{tile}")


# -------------------------------------------------- paper-fixed behaviour --

def test_hand_worked_cases_on_gpu():
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_4x4.json")))
    for case in g["cases"]:
        shape = tuple(case["shape"])
        phi = np.zeros(shape)
        if "impulse" in case:
            phi[tuple(reversed(case["impulse"]))] = 1.0
        else:
            phi[...] = case["uniform"]
        expect = np.zeros(shape)
        if "expect_all" in case:
            expect[...] = case["expect_all"]
        for key, val in case.get("expect", {}).items():
            expect[tuple(reversed(json.loads(key)))] = val
        for variant, k, tile in schedules(len(shape), "f64"):
            out = gpu_run(phi, g["h"], g["eps"], g["dt"], 1, "f64", variant, k, tile)
            np.testing.assert_allclose(out, expect, rtol=0, atol=1e-15, err_msg=case["name"])


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("shape", [(40, 70), (9, 20, 30)])
def test_fixed_points_bitwise_on_gpu(shape, dtype):
    h, eps, dt = _params(shape)
    for value in (1.0, -1.0, 0.0):
        phi0 = np.full(shape, value)
        for variant, k, tile in schedules(len(shape), dtype):
            out = gpu_run(phi0, h, eps, dt, 2 * k + 3, dtype, variant, k, tile)
            assert np.array_equal(out, phi0), f"value {value} v{variant} k{k} t{tile}"


def test_mirror_symmetry_on_gpu_fp64():
    # grid mirror symmetry holds bit for bit on the GPU path as well
    shape = (48, 48)
    h, eps, dt = _params(shape)
    phi0 = wl.random_field(shape, seed=9)
    for variant, k, tile in schedules(2, "f64"):
        a = gpu_run(phi0, h, eps, dt, 12, "f64", variant, k, tile)
        b = gpu_run(phi0[:, ::-1].copy(), h, eps, dt, 12, "f64", variant, k, tile)
        c = gpu_run(phi0.T.copy(), h, eps, dt, 12, "f64", variant, k, tile)
        assert np.array_equal(a[:, ::-1], b)
        assert np.array_equal(a.T, c)


def test_mirror_symmetry_3d_every_tile():
    # x/y/z mirrors and the x<->y swap of a cube commute with every 3D
    # schedule and tile bit for bit (paired neighbour sums)
    shape = (12, 40, 40)
    h, eps, dt = _params(shape)
    phi0 = wl.random_field(shape, seed=4)
    for variant, k, tile in schedules(3, "f32"):
        a = gpu_run(phi0, h, eps, dt, 2 * k + 1, "f32", variant, k, tile)
        for f, inv in ((lambda x: x[:, :, ::-1], lambda x: x[:, :, ::-1]),
                       (lambda x: x[:, ::-1, :], lambda x: x[:, ::-1, :]),
                       (lambda x: x[::-1], lambda x: x[::-1]),
                       (lambda x: x.transpose(0, 2, 1), lambda x: x.transpose(0, 2, 1))):
            b = gpu_run(np.ascontiguousarray(f(phi0)), h, eps, dt, 2 * k + 1, "f32", variant, k, tile)
            assert np.array_equal(inv(b), a), f"v{variant} k{k} t{tile}"


@pytest.mark.parametrize("dtype", ["f32", "f16s"])
def test_axis_invariance_every_schedule(dtype):
    # a field constant along one axis stays constant along it bit for bit:
    # tile, strip, chunk and halo seams along that axis, and the faces across
    # it, must not leak into the result
    for shape in ((70, 530), (10, 70, 260)):
        nd = len(shape)
        h, eps, dt = _params(shape)
        for axis in range(nd):
            base = tuple(1 if a == axis else shape[a] for a in range(nd))
            phi0 = np.repeat(wl.random_field(base, seed=axis), shape[axis], axis=axis)
            for variant, k, tile in schedules(nd, dtype):
                a = gpu_run(phi0, h, eps, dt, 2 * k + 1, dtype, variant, k, tile)
                ref = np.take(a, [0], axis=axis)
                assert np.array_equal(a, np.broadcast_to(ref, a.shape)), \
                    f"{shape} axis {axis} v{variant} k{k} t{tile}"


def test_tile_selection_api():
    sim2 = ac.Simulation((16, 16), 1 / 16, 0.1, 1e-4, dtype="f32")
    sim3 = ac.Simulation((8, 16, 16), 1 / 16, 0.1, 1e-4, dtype="f32")
    sim2h = ac.Simulation((16, 16), 1 / 16, 0.1, 1e-4, dtype="f16s")
    big = ac.Simulation((4096, 4096), 1 / 4096, 4 / 4096, 0.1 / 4096 ** 2, dtype="f32")
    mid = ac.Simulation((1024, 1024), 1 / 1024, 4 / 1024, 0.1 / 1024 ** 2, dtype="f32")
    try:
        assert sim2.tile() == 0 and sim2.schedule() == (ac.AC_VARIANT_STREAM, 4)
        assert big.tile() == 1 and big.schedule() == (ac.AC_VARIANT_STREAM, 6)  # 8-cell strips from 4096^2
        assert mid.tile() == 0 and mid.schedule() == (ac.AC_VARIANT_STREAM, 5)  # 4-cell strips, k = 5
        sim2.set_tile(0)
        sim2.set_tile(1)             # FP32 2D: strips of 8 cells per lane
        assert sim2.tile() == 1
        with pytest.raises(ac.AcError) as e:
            sim2.set_tile(ac.AC_NUM_TILES_2D)
        assert e.value.code == ac.AC_ERR_INVALID
        with pytest.raises(ac.AcError) as e:
            sim2h.set_tile(1)        # FP16 storage has one strip width
        assert e.value.code == ac.AC_ERR_UNSUPPORTED
        with pytest.raises(ac.AcError) as e:
            sim3.set_tile(ac.AC_NUM_TILES_3D)
        assert e.value.code == ac.AC_ERR_INVALID
        for t in range(ac.AC_NUM_TILES_3D):
            sim3.set_tile(t)
            assert sim3.tile() == t
        sim3.set_schedule(ac.AC_VARIANT_DIRECT, 1)
        assert sim3.tile() == 0      # the direct kernel has no tiles
        sim3.set_schedule(ac.AC_VARIANT_AUTO, 0)
        sim3.set_tile(ac.AC_TILE_AUTO)
        assert sim3.tile() in range(ac.AC_NUM_TILES_3D)
    finally:
        big.close()
        mid.close()
        sim2h.close()
        sim2.close()
        sim3.close()


def test_fp16_error_report_against_fp64():
    # FP16 storage with FP32 arithmetic: rounding happens once per pass of k
    # steps, so deeper temporal blocking is at least as accurate
    w = wl.CIRCLE_64
    phi0 = oracle.init_sphere(w.shape, w.h, w.r0, w.eps)
    ref = oracle.step(phi0, w.h, w.eps, w.dt, w.steps)
    errs = {}
    for variant, k, tile in schedules(2, "f16s"):
        out = gpu_run(phi0, w.h, w.eps, w.dt, w.steps, "f16s", variant, k, tile)
        errs[(variant, k)] = (rel_l2(out, ref), float(np.max(np.abs(out - ref))))
        assert errs[(variant, k)][0] <= 1e-3
    assert errs[(2, 6)][0] <= errs[(2, 1)][0] * 1.05
