"""Contexts driven from several host threads at once: each kernel's one-time,
per-device set-up (shared-memory limit, occupancy) is taken under a lock, so
concurrent first launches must all succeed and give the same fields as the
same work done one context at a time."""
import threading

import numpy as np
import pytest

import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# (shape, dtype, k, tile): distinct kernels, so several first launches race
CASES = [((20, 24, 40), "f32", 1, 1), ((20, 24, 40), "f32", 3, 2), ((33, 17, 64), "f16s", 2, 1),
         ((96, 136), "f32", 5, 1), ((96, 136), "f16s", 3, 0), ((17, 20, 24), "f64", 2, 2)]


def _run(shape, dtype, k, tile, out, i, barrier):
    import torch
    h = 1.0 / max(shape)
    sim = ac.Simulation(shape, h, 3 * h, 0.1 * h * h, dtype=dtype, stream=torch.cuda.Stream())
    try:
        sim.load(wl.smooth_field(shape, seed=i))
        sim.set_schedule(ac.AC_VARIANT_STREAM, k)
        sim.set_tile(tile)
        if barrier is not None:
            barrier.wait()
        sim.step(2 * k + 1)
        assert sim.status() == ac.AC_OK
        out[i] = sim.to_numpy()
    finally:
        sim.close()


def test_concurrent_first_launches_from_threads():
    par = [None] * len(CASES)
    barrier = threading.Barrier(len(CASES))
    errors = []

    def worker(i):
        try:
            _run(*CASES[i], par, i, barrier)
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(CASES))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not errors, errors
    seq = [None] * len(CASES)
    for i, c in enumerate(CASES):
        _run(*c, seq, i, None)
    for i in range(len(CASES)):
        assert np.array_equal(par[i], seq[i]), f"case {i}"
