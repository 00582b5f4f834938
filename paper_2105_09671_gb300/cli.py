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
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--eps-cells", type=float, default=1.5, help="eps in units of h")
    ap.add_argument("--init", default="sphere", choices=["sphere", "random"])
    ap.add_argument("--autotune", action="store_true")
    args = ap.parse_args(argv)

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
    if args.init == "sphere":
        sim.init_sphere(r0=0.25)
    else:
        sim.init_random(seed=0)
    if args.autotune:
        sim.autotune()
    v, k = sim.schedule()
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
    print(json.dumps({"shape": list(shape), "dtype": args.dtype, "variant": v, "k": k,
                      "steps": args.steps, "ms": best,
                      "gcell_updates_per_s": cells * args.steps / (best / 1e3) / 1e9,
                      "energy": energy, "status": sim.status()}))
    sim.close()


if __name__ == "__main__":
    main()
