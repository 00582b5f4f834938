"""The allocation-free observation entry point, ac_observe_noalloc.

Some callers cannot allocate at the moment they want the energy of a field:
their device memory belongs to another allocator or a fixed budget, or they
sit in a latency-critical loop that cannot take the device-wide
synchronisation of cudaMalloc/cudaFree.  ac_observe_noalloc serves them from
a fixed array compiled into the library.  These tests call it through the C
ABI and compare it with ac_observe, which works from a context's own buffers.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import _lib as L
from paper_2105_09671_gb300 import workloads as wl


def test_rejects_grids_beyond_the_scratch_limit():
    # 2048 x 1024 rows is twice the fixed scratch; refused before any CUDA call
    d = ac.make_desc(3, ac.AC_F32, 8, 2048, 1024, 8, 1 / 2048, 0.01, 1e-8)
    rc = ac.lib().ac_observe_noalloc(ctypes.byref(d), ctypes.c_void_p(0x10000), None,
                                     ctypes.c_void_p(0x20000))
    assert rc == ac.AC_ERR_INVALID
    assert "scratch limit" in L.last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,shape", [("f32", (300, 257)), ("f64", (31, 40, 77)),
                                         ("f16s", (64, 64)), ("f32", (512, 512, 512)),
                                         # exactly at the limit: ny * nz = 1048576 rows, so
                                         # the last of the 16384 partial slots is used
                                         ("f32", (1024, 1024, 8))])
def test_matches_context_observe_on_two_calls(dtype, shape):
    import torch

    h = 1.0 / max(shape)
    eps = 3 * h
    sim = ac.Simulation(shape, h, eps, 0.1 * h * h, dtype=dtype)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=sim.device)
    try:
        for call in range(2):
            if call == 0:
                if shape == (512, 512, 512):
                    sim.init_sphere(r0=0.25)
                else:
                    sim.load(wl.smooth_field(shape, seed=5))
            else:
                sim.step(7)  # a different field: nothing may carry over between calls
            ref = sim.observe()
            ac.ac_observe_noalloc(sim.desc, sim._buf.data_ptr(), sim.stream.cuda_stream,
                                  out.data_ptr())
            sim.stream.synchronize()
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(ref[0], rel=1e-12), f"call {call}: energy"
            assert got[1] == pytest.approx(ref[1], rel=1e-12), f"call {call}: volume"
            assert got[2] == ref[2] == 0.0
    finally:
        sim.close()


@pytest.mark.gpu
def test_counts_nonfinite_cells_like_the_context_path():
    import torch

    shape = (33, 40)
    sim = ac.Simulation(shape, 1 / 40, 0.1, 0.1 / 1600, dtype="f32")
    out = torch.zeros(3, dtype=torch.float64, device=sim.device)
    try:
        a = np.zeros(shape)
        a[3, 7] = np.nan
        a[20, 39] = np.inf
        sim.load(a)
        ref = sim.observe(allow_nonfinite=True)
        for _ in range(2):
            ac.ac_observe_noalloc(sim.desc, sim._buf.data_ptr(), sim.stream.cuda_stream,
                                  out.data_ptr())
            sim.stream.synchronize()
            assert out[2].item() == ref[2] == 2.0
    finally:
        sim.close()
