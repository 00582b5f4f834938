"""Slab decomposition on the CPU: the plan (host arithmetic of the C
library, no CUDA call) and the multi-rank halo exchange of DistributedSlab
over gloo ranks, each rank advancing its extended slab with the FP64
oracle.  The decomposed run must equal the undivided oracle run bit for
bit: a cell's update reads only its neighbours, so with fresh halos every
owned cell sees exactly the inputs it sees in the whole grid."""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_2105_09671_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("extent,parts,halo", [(512, 8, 4), (100, 3, 8), (17, 2, 8), (9, 9, 1),
                                               (5, 1, 16), (130, 4, 16)])
def test_plan_partitions_the_axis(extent, parts, halo):
    plan = L.ac_slab_plan(extent, parts, halo)
    assert len(plan) == parts
    sizes = [hi - lo for lo, hi, _, _ in plan]
    assert plan[0][0] == 0 and plan[-1][1] == extent
    assert all(plan[p][1] == plan[p + 1][0] for p in range(parts - 1))  # contiguous, no overlap
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    for p, (lo, hi, elo, ehi) in enumerate(plan):
        assert elo == (lo - halo if p > 0 else 0)
        assert ehi == (hi + halo if p + 1 < parts else extent)
        if parts > 1:
            assert hi - lo >= halo  # every halo comes from one neighbour


@pytest.mark.parametrize("extent,parts,halo", [(8, 9, 1), (0, 1, 1), (10, 0, 1), (10, 2, 0),
                                               (15, 2, 8)])
def test_plan_rejects_impossible_splits(extent, parts, halo):
    with pytest.raises(L.AcError) as e:
        L.ac_slab_plan(extent, parts, halo)
    assert e.value.code == L.AC_ERR_INVALID


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import oracle
from paper_2105_09671_gb300 import workloads as wl
from paper_2105_09671_gb300.slab import DistributedSlab

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
shape, halo, nsteps = {shape!r}, {halo}, {nsteps}
n = max(shape)
h = 1.0 / n
eps, dt = 3.0 * h, 0.1 * h * h
phi0 = wl.smooth_field(shape, seed=11) + 0.05 * np.random.default_rng(2).uniform(-1, 1, shape)
from paper_2105_09671_gb300.slab import plan
own_lo, own_hi, ext_lo, ext_hi = plan(shape[0], world, halo)[rank]
field = torch.from_numpy(phi0[ext_lo:ext_hi].copy())
steps_taken = []
def step_fn(b):
    steps_taken.append(b)
    field.copy_(torch.from_numpy(oracle.step(field.numpy(), h, eps, dt, b)))
ds = DistributedSlab(shape[0], halo, field, step_fn)
ds.mark_fresh()
ds.step(nsteps)
parts = [None] * world
dist.all_gather_object(parts, ds.owned().numpy())
if rank == 0:
    got = np.concatenate(parts, axis=0)
    ref = oracle.step(phi0, h, eps, dt, nsteps)
    print(json.dumps({{"equal": bool(np.array_equal(got, ref)), "maxabs": float(np.max(np.abs(got - ref))),
                       "blocks": steps_taken, "exchanges": ds.exchanges}}), flush=True)
else:
    print(json.dumps({{"blocks": steps_taken, "exchanges": ds.exchanges}}), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,shape,halo,nsteps", [
    (2, (40, 33), 4, 19),          # 2D, split in y, a remainder block of 3 steps
    (3, (37, 24), 8, 40),          # 2D, uneven parts (13, 12, 12)
    (2, (21, 12, 10), 3, 10),      # 3D, split in z
    (3, (30, 9, 11), 5, 23),       # 3D, three parts, remainder
])
def test_gloo_ranks_reproduce_the_undivided_run(world, shape, halo, nsteps):
    port = _free_port()
    code = RANK_SCRIPT.format(root=ROOT, shape=shape, halo=halo, nsteps=nsteps)
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
               CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, "-c", code], env=dict(env, RANK=str(r), LOCAL_RANK=str(r)),
                              cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    res = outs[0]
    assert res["equal"], f"max-abs {res['maxabs']}"
    blocks = [halo] * (nsteps // halo) + ([nsteps % halo] if nsteps % halo else [])
    for o in outs:
        assert o["blocks"] == blocks
        assert o["exchanges"] == len(blocks) - 1  # halos fresh at the start
