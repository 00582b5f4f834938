"""Command-line runner: advance one grid on the GPU and report timing.

    python -m paper_2105_09671_gb300.cli --shape 512 512 192 --dtype f32 --k 2 --steps 8

Creates the grid with a device-side sphere (or random) initial state, runs
``--steps`` Euler steps through ac_step with the requested schedule, prints
the elapsed time (CUDA events), Gcell-updates/s and the energy.  Used for
profiling single kernels on cases of a chosen size.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    import torch

    import paper_2105_09671_gb300 as ac

    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", type=int, nargs="+", required=True, help="ny nx or nz ny nx")
    ap.add_argument("--dtype", default="f32", choices=["f64", "f32", "f16s"])
    ap.add_argument("--k", type=int, default=0, help="temporal depth; -1 = direct kernel; 0 = default")
    ap.add_argument("--tile", type=int, default=-1, help="3D streaming tile; -1 = default")
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--eps-cells", type=float, default=1.5, help="eps in units of h")
    ap.add_argument("--init", default="sphere", choices=["sphere", "random"])
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--graph", action="store_true", help="replay the steps as one CUDA graph")
    ap.add_argument("--net", action="store_true",
                    help="run the learned jump network forward instead of the stepper")
    args = ap.parse_args(argv)
    if args.net:
        return net_main(args)

    shape = tuple(args.shape)
    h = 1.0 / shape[-1]
    eps = args.eps_cells * h
    dt = 0.1 * h * h
    stream = torch.cuda.Stream()
    sim = ac.Simulation(shape, h, eps, dt, dtype=args.dtype, stream=stream)
    if args.k > 0:
        sim.set_schedule(ac.AC_VARIANT_STREAM, args.k)
    elif args.k < 0:
        sim.set_schedule(ac.AC_VARIANT_DIRECT, 1)
    if args.tile >= 0:
        sim.set_tile(args.tile)
    if args.init == "sphere":
        sim.init_sphere(r0=0.25)
    else:
        sim.init_random(seed=0)
    if args.graph:
        sim.set_graph(True)  # before autotuning: candidates are then timed as graphs
    if args.autotune:
        sim.autotune()
    if args.graph:
        sim.step(args.steps)  # the capture, outside the timed runs
        stream.synchronize()
    v, k = sim.schedule()
    tile = sim.tile()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.repeat):
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        stream.synchronize()
        times.append(e0.elapsed_time(e1))
    energy = sim.energy()
    cells = 1
    for s in shape:
        cells *= s
    best = min(times)
    print(json.dumps({"shape": list(shape), "dtype": args.dtype, "variant": v, "k": k, "tile": tile,
                      "graph": bool(args.graph), "steps": args.steps, "ms": best,
                      "gcell_updates_per_s": cells * args.steps / (best / 1e3) / 1e9,
                      "energy": energy, "status": sim.status()}))
    sim.close()


def net_main(args):
    """Forward passes of the jump network (He-initialised, seed 0) on a random
    field of the given shape; prints the mean time per forward."""
    import torch

    from paper_2105_09671_gb300 import _lib as L

    shape = tuple(args.shape)
    ndim = len(shape)
    stream = torch.cuda.Stream()
    net = L.ac_net_create(ndim, stream.cuda_stream)
    x = torch.rand(shape, device="cuda") * 2 - 1
    y = torch.empty_like(x)
    nz = shape[0] if ndim == 3 else 1
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        L.ac_net_forward(net, x.data_ptr(), y.data_ptr(), 1, shape[-1], shape[-2], nz, 0.1)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cells = 1
    for v in shape:
        cells *= v
    print(json.dumps({"shape": list(shape), "forward_ms": ms,
                      "mcells_per_s": cells / (ms / 1e3) / 1e6}))
    L.ac_net_destroy(net)


if __name__ == "__main__":
    main()
