"""The batched persistent stepper against the single-grid stepper and the
oracle, plus its graph replay and its bounded-wait timeout path."""
import numpy as np
import pytest

import oracle
import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

from gpu_util import NP, assert_parity, stored

pytestmark = pytest.mark.gpu


def _specs(shapes, seed=0):
    rng = np.random.default_rng(seed)
    specs, inits = [], []
    for i, shp in enumerate(shapes):
        h = 1.0 / max(shp)
        eps = float(rng.uniform(3, 6)) * h
        specs.append((shp, h, eps, 0.1 * h * h))
        if i % 2:
            inits.append(oracle.init_random(shp, seed=100 + i))
        else:
            inits.append(oracle.init_sphere(shp, h, float(rng.uniform(0.1, 0.4)), eps))
    return specs, inits


SHAPES = [(1, 1), (3, 130), (64, 64), (97, 33), (130, 250), (200, 121), (257, 257), (40, 300)]


BATCH_SCHEDULES = [(d, k, 0) for d in ("f32", "f64", "f16s") for k in (1, 2, 3, 4)] + \
    [("f32", k, 1) for k in (1, 2, 3, 4, 5, 6)]


@pytest.mark.parametrize("dtype,k,tile", BATCH_SCHEDULES)
def test_batch_equals_single_grid_stepper_bitwise(dtype, k, tile):
    specs, inits = _specs(SHAPES, seed=k)
    n = [5, 0, 1, 2 * k + 1, 37, 64, 13, 9]
    b = ac.Batch(specs, dtype=dtype)
    try:
        b.set_tile(tile)
        b.set_schedule(k)
        assert b.tile() == tile
        for i, a in enumerate(inits):
            b.load(i, a)
        b.step(n)
        assert b.status() == ac.AC_OK
        got = [b.to_numpy(i) for i in range(len(b))]
    finally:
        b.close()
    for i, (spec, a) in enumerate(zip(specs, inits)):
        shp, h, eps, dt = spec
        sim = ac.Simulation(shp, h, eps, dt, dtype=dtype)
        try:
            sim.load(a)
            sim.set_schedule(ac.AC_VARIANT_STREAM, min(k, 8))
            sim.step(n[i])
            ref = sim.to_numpy()
        finally:
            sim.close()
        assert np.array_equal(got[i], ref), f"instance {i} {shp} n={n[i]}"
        o = oracle.step(stored(a, dtype), h, eps, dt, n[i])
        assert_parity(got[i].astype(np.float64), o, dtype, f"instance {i} vs oracle")


def test_batch_tile_selection_api():
    specs, _ = _specs(SHAPES[2:4], seed=1)
    b32 = ac.Batch(specs, dtype="f32")
    b16 = ac.Batch(specs, dtype="f16s")
    try:
        assert b32.tile() == 0
        with pytest.raises(ac.AcError) as e:
            b32.set_schedule(5)          # depth 5 needs the 8-cell strips
        assert e.value.code == ac.AC_ERR_INVALID
        b32.set_tile(1)
        b32.set_schedule(6)
        with pytest.raises(ac.AcError) as e:
            b32.set_tile(0)              # depth 6 is not offered with tile 0
        assert e.value.code == ac.AC_ERR_UNSUPPORTED
        with pytest.raises(ac.AcError) as e:
            b16.set_tile(1)
        assert e.value.code == ac.AC_ERR_UNSUPPORTED
    finally:
        b16.close()
        b32.close()


def test_batch_uneven_workload_2000_steps_against_oracle():
    # the batched workload's kind of instances: sizes 64..1024, eps 3h..6h,
    # random and circle states, 2000 steps, FP32; compared with the FP64 oracle
    shapes = [(64, 64), (160, 160), (352, 352), (608, 608), (1024, 1024)]
    specs, inits = _specs(shapes, seed=7)
    b = ac.Batch(specs, dtype="f32")
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        b.step(2000)
        assert b.status() == ac.AC_OK
        got = [b.to_numpy(i).astype(np.float64) for i in range(len(b))]
    finally:
        b.close()
    for i, (spec, a) in enumerate(zip(specs, inits)):
        shp, h, eps, dt = spec
        o = oracle.step(stored(a, "f32"), h, eps, dt, 2000)
        rel = float(np.linalg.norm(got[i] - o) / np.linalg.norm(o))
        assert rel <= 1e-3, f"instance {i}: rel-L2 {rel:.2e}"
        assert float(np.max(np.abs(got[i] - o))) <= 1e-4


def test_batched_workload_sampled_instances_against_oracle():
    # the batched workload itself: 512 uneven grids (64^2 .. 1024^2, eps 3h..6h,
    # circles and random states), autotuned depth, graph-replayed, 2000 steps;
    # 16 instances drawn at random are compared with the FP64 oracle
    import torch
    inst = wl.batch_instances(512, seed=0)
    specs = [((d["n"], d["n"]), d["h"], d["eps"], d["dt"]) for d in inst]
    inits = []
    for d in inst:
        shp = (d["n"], d["n"])
        inits.append(oracle.init_sphere(shp, d["h"], d["r0"], d["eps"]) if d["init"] == "sphere"
                     else oracle.init_random(shp, seed=d["seed"]))
    s = torch.cuda.Stream()
    b = ac.Batch(specs, dtype="f32", stream=s)
    sample = np.random.default_rng(2024).choice(len(inst), size=16, replace=False)
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        b.autotune(64)  # restores the fields it times on
        k, tile = b.schedule(), b.tile()
        assert 1 <= k <= (4 if tile == 0 else 6)
        b.set_graph(True)
        b.step(2000)
        assert b.status() == ac.AC_OK
        got = {int(i): b.to_numpy(int(i)).astype(np.float64) for i in sample}
    finally:
        b.close()
    worst = 0.0
    for i in sample:
        d = inst[int(i)]
        o = oracle.step(stored(inits[int(i)], "f32"), d["h"], d["eps"], d["dt"], 2000)
        rel = float(np.linalg.norm(got[int(i)] - o) / np.linalg.norm(o))
        worst = max(worst, rel)
        assert rel <= 1e-3, f"instance {i} (n = {d['n']}): rel-L2 {rel:.2e}"
        assert float(np.max(np.abs(got[int(i)] - o))) <= 1e-4
    print(f"\nbatch512: autotuned k = {k}, tile {tile}; 16 sampled instances, worst rel-L2 {worst:.2e}")


def test_batch_graph_replay_and_launch_count():
    import torch
    specs, inits = _specs(SHAPES[2:6], seed=3)
    s = torch.cuda.Stream()
    b = ac.Batch(specs, dtype="f32", stream=s)
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        b.set_graph(True)
        c0 = b.launch_count()
        for _ in range(3):
            b.step(10)
        assert b.launch_count() - c0 == 3  # one persistent kernel per call
        got = [b.to_numpy(i).astype(np.float64) for i in range(len(b))]
    finally:
        b.close()
    for i, (spec, a) in enumerate(zip(specs, inits)):
        shp, h, eps, dt = spec
        assert_parity(got[i], oracle.step(stored(a, "f32"), h, eps, dt, 30), "f32", f"graph {i}")


def test_batch_bounded_wait_times_out_and_recovers():
    # one-poll waits give up as soon as a neighbour is not already done: the
    # kernel reports AC_ERR_TIMEOUT instead of waiting; nothing hangs and the
    # batch works again with the default limit
    specs, inits = _specs([(512, 512), (300, 700)], seed=5)
    b = ac.Batch(specs, dtype="f32")
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        b.set_wait_limit(1)
        b.step(64)
        assert b.status() == ac.AC_ERR_TIMEOUT
        b.set_wait_limit(0)
        for i, a in enumerate(inits):
            b.load(i, a)
        b.step(8)
        assert b.status() == ac.AC_OK
        got = b.to_numpy(1).astype(np.float64)
    finally:
        b.close()
    shp, h, eps, dt = specs[1]
    assert_parity(got, oracle.step(stored(inits[1], "f32"), h, eps, dt, 8), "f32", "after timeout")


def test_batch_observe_matches_oracle():
    specs, inits = _specs(SHAPES[2:5], seed=11)
    b = ac.Batch(specs, dtype="f64")
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        for i, (spec, a) in enumerate(zip(specs, inits)):
            e, v, bad = b.observe(i)
            assert e == pytest.approx(oracle.energy(a, spec[1], spec[2]), rel=1e-12)
            assert v == pytest.approx(oracle.phase_volume(a, spec[1]), rel=1e-12)
            assert bad == 0
    finally:
        b.close()


def test_batch_autotune_keeps_fields():
    specs, inits = _specs(SHAPES[2:5], seed=2)
    b = ac.Batch(specs, dtype="f32")
    try:
        for i, a in enumerate(inits):
            b.load(i, a)
        b.autotune(16)
        assert 1 <= b.schedule() <= 4
        for i, a in enumerate(inits):
            assert np.array_equal(b.to_numpy(i), a.astype(np.float32))
    finally:
        b.close()
