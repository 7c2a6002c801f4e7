"""Reconstruct synthetic captures of a named workload through the C ABI.

    python -m paper_2608_28183_gb300.run --workload pf_128x128x1024 --steps 5 [--storage f16]
        [--tune-cache path.json] [--grid NX,NY,NT]

Prints one line per run with the per-stage CUDA-event times. Meant for
profiling captures and quick checks; the benchmark is bench.py at the
repository root.
"""
from __future__ import annotations

import argparse
import json
import os


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="fk_256x256x512",
                    choices=["fk_32x32x256", "pf_128x128x1024", "fk_256x256x512"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--grid", default=None, help="nx,ny,nt override (same scene recipe)")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args(argv)

    import torch
    from . import build, nlos, synth
    build.build()
    geom = None
    if args.grid:
        nx, ny, nt = (int(v) for v in args.grid.split(","))
        spec = synth.WORKLOADS[args.workload]["geom"]
        geom = synth.Geometry(nx, ny, nt, spec.bin_width_s, spec.wall_w_m, spec.wall_h_m)
    cap = synth.make_capture(args.workload, 0, device="cuda", geom=geom)
    g = cap.geometry
    kw = {}
    method = "pf" if args.workload.startswith("pf") else "fk"
    if method == "pf":
        kw = dict(n_depths=128, depth_min_m=0.5, depth_max_m=2.5)
    plan = nlos.plan_for_capture(g, method, args.storage, **kw)
    if not args.no_autotune:
        plan.autotune()
    x = torch.as_tensor(cap.counts, dtype=torch.float32).to(plan.input_dtype()).cuda()
    v = plan.empty_volume()
    plan.set_profiling(True)
    for _ in range(args.steps):
        plan.reconstruct(x, v)
    torch.cuda.synchronize()
    stages, calls = plan.stage_times()
    print(json.dumps({"workload": args.workload, "grid": [g.nx, g.ny, g.nt], "storage": args.storage,
                      "tiles": plan.tiles, "calls": calls,
                      "stages_ms": {k: val / max(1, calls) for k, val in stages.items()}}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
