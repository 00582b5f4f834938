"""Schedules on the GPU: the autotuner leaves the field untouched and picks a
schedule the library offers, the tuned choice is reused per size class, and
graph replay re-captures when the schedule or the tile changes."""
import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import assert_parity, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,dtype", [((48, 64, 80), "f32"), ((130, 200), "f32"),
                                         ((24, 40, 48), "f64"), ((40, 72, 96), "f16s")])
def test_autotune_keeps_field_and_steps_correctly(shape, dtype):
    import torch
    h = 1.0 / max(shape)
    eps, dt = 2.5 * h, 0.1 * h * h
    phi0 = wl.smooth_field(shape, seed=11) + 0.05 * wl.random_field(shape, seed=12)
    s = torch.cuda.Stream()
    sim = ac.Simulation(shape, h, eps, dt, dtype=dtype, stream=s)
    try:
        sim.load(phi0)
        before = sim.to_numpy().copy()
        sim.autotune(8)
        assert np.array_equal(sim.to_numpy(), before), "autotune changed the field"
        v, k = sim.schedule()
        tile = sim.tile()
        assert v in (ac.AC_VARIANT_DIRECT, ac.AC_VARIANT_STREAM) and 1 <= k <= ac.AC_MAX_K
        assert 0 <= tile < (ac.AC_NUM_TILES_3D if len(shape) == 3 else ac.AC_NUM_TILES_2D)
        sim.step(23)
        assert sim.status() == ac.AC_OK
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    assert_parity(out, oracle_run(phi0, h, eps, dt, 23, dtype), dtype, f"tuned v{v} k{k} t{tile}")
    # a second context of the same size class reuses the cached choice
    sim2 = ac.Simulation(shape, h, eps, dt, dtype=dtype, stream=s)
    try:
        sim2.autotune(8)
        assert sim2.schedule() == (v, k) and sim2.tile() == tile
    finally:
        sim2.close()


def test_graph_replay_recaptures_on_schedule_and_tile_change():
    import torch
    shape = (20, 36, 44)
    h = 1.0 / 44
    eps, dt = 2.5 * h, 0.1 * h * h
    phi0 = wl.smooth_field(shape, seed=5)
    s = torch.cuda.Stream()
    sim = ac.Simulation(shape, h, eps, dt, dtype="f32", stream=s)
    try:
        sim.load(phi0)
        sim.set_graph(True)
        n0 = sim.launch_count()
        sim.set_schedule(ac.AC_VARIANT_STREAM, 2)
        sim.set_tile(0)
        sim.step(6)
        sim.step(6)                 # replay
        sim.set_tile(2)
        sim.step(6)                 # re-captured with tile 2
        sim.set_schedule(ac.AC_VARIANT_DIRECT, 1)
        sim.step(6)                 # re-captured with the direct kernel
        assert sim.status() == ac.AC_OK
        # 6 steps at depth 2 are launched as 2 + 2 + 1 + 1 (an even count
        # ends the result in phi), then 6 direct launches
        assert sim.launch_count() - n0 == 4 + 4 + 4 + 6
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    assert_parity(out, oracle_run(phi0, h, eps, dt, 24, "f32"), "f32", "graph sequence")


def test_tune_cache_file_round_trip(tmp_path):
    import torch
    path = tmp_path / "tune.txt"
    shape = (24, 40, 48)
    h = 1.0 / 48
    eps, dt = 2.5 * h, 0.1 * h * h
    s = torch.cuda.Stream()
    ac.ac_set_tune_cache(str(path))
    try:
        sim = ac.Simulation(shape, h, eps, dt, dtype="f32", stream=s)
        try:
            sim.autotune(4)
            tuned = (sim.schedule(), sim.tile())
        finally:
            sim.close()
        lines = path.read_text().splitlines()
        assert len(lines) == 1
        tag, nd, dt_code, cls, dev, gr, v, k, t = lines[0].split()
        assert tag == "ac-tune-v2" and int(nd) == 3 and int(dt_code) == ac.AC_F32 and int(gr) == 0
        assert (int(v), int(k)) == tuned[0] and int(t) == tuned[1]
        # a later entry for the same key wins: a new process (emulated by
        # emptying the process cache) adopts it without timing; an entry of
        # the earlier v1 form (no graph field) counts as timed without graphs,
        # and an entry for graph replay does not apply to this context
        other = (ac.AC_VARIANT_DIRECT, 1, 0) if tuned[0][0] == ac.AC_VARIANT_STREAM \
            else (ac.AC_VARIANT_STREAM, 1, 0)
        third = (ac.AC_VARIANT_STREAM, 2, 2)
        with open(path, "a") as f:
            f.write(f"ac-tune-v1 {nd} {dt_code} {cls} {dev} {other[0]} {other[1]} {other[2]}\n")
            f.write(f"ac-tune-v2 {nd} {dt_code} {cls} {dev} 1 {third[0]} {third[1]} {third[2]}\n")
            f.write("not a cache line\n")
        ac.ac_set_tune_cache(str(path))
        sim = ac.Simulation(shape, h, eps, dt, dtype="f32", stream=s)
        try:
            n0 = sim.launch_count()
            sim.autotune(4)
            assert sim.launch_count() == n0  # nothing was timed
            assert sim.schedule() == other[:2] and sim.tile() == other[2]
        finally:
            sim.close()
        ac.ac_set_tune_cache(str(path))
        sim = ac.Simulation(shape, h, eps, dt, dtype="f32", stream=s)
        try:
            sim.set_graph(True)  # the graph-replay entry applies now
            n0 = sim.launch_count()
            sim.autotune(4)
            assert sim.launch_count() == n0
            assert sim.schedule() == third[:2] and sim.tile() == third[2]
        finally:
            sim.close()
    finally:
        ac.ac_set_tune_cache(None)


def test_autotune_with_graph_replay_times_graphs():
    # a small grid is bound by launch overhead; with graph replay on, the
    # candidates are timed as replayed graphs (the field is kept) and the
    # choice is cached apart from the one timed as launches
    import torch
    shape = (64, 64)
    h = 1.0 / 64
    eps, dt = 0.015, 0.1 * h * h
    phi0 = wl.smooth_field(shape, seed=3)
    s = torch.cuda.Stream()
    ac.ac_set_tune_cache(None)
    sim = ac.Simulation(shape, h, eps, dt, dtype="f64", stream=s)
    try:
        sim.load(phi0)
        before = sim.to_numpy().copy()
        sim.set_graph(True)
        sim.autotune(32)
        assert np.array_equal(sim.to_numpy(), before)
        v, k = sim.schedule()
        sim.step(40)
        assert sim.status() == ac.AC_OK
        out = sim.to_numpy().astype(np.float64)
    finally:
        sim.close()
    assert_parity(out, oracle_run(phi0, h, eps, dt, 40, "f64"), "f64", f"graph-tuned v{v} k{k}")
