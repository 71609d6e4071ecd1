"""Run the FLBM step on one channel configuration and print per-kernel times.

    python -m paper_1909_01092_gb300.run --lx 128 --ly 128 --lz 128 --kT 1e-5 --radius 12 --steps 20

Defaults are the 128x128x512 fluctuating channel with the R=12 sphere. The
output is one JSON line: MLUPS of the timed steps and the CUDA-event time of
each kernel class per step. Useful for profiler captures of a chosen case.

    python -m paper_1909_01092_gb300.run --lx 64 --ly 64 --lz 128 --kT 0 --radius 8 --delta-rho 0.3 \
        --adjoint 20 --checkpoint-every 10

runs the adjoint of that many steps instead (J, gradient, milliseconds), and

    python -m paper_1909_01092_gb300.run --ensemble 128 --steps 4

steps the uneven 128-replica ensemble with a fixed launch configuration.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--lx", type=int, default=128)
    ap.add_argument("--ly", type=int, default=128)
    ap.add_argument("--lz", type=int, default=512)
    ap.add_argument("--kT", type=float, default=1e-5)
    ap.add_argument("--radius", type=float, default=12.0)
    ap.add_argument("--g", type=float, default=1e-5)
    ap.add_argument("--G", type=float, default=1.2)
    ap.add_argument("--delta-rho", type=float, default=0.0)
    ap.add_argument("--walls", default="xy", help="walled axes, e.g. xy, xyz or none")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--adjoint", type=int, default=0, help="adjoint of this many noise-free steps")
    ap.add_argument("--checkpoint-every", type=int, default=100)
    ap.add_argument("--ensemble", type=int, default=0, help="step this many ensemble replicas instead")
    a = ap.parse_args(argv)

    import torch

    from . import binding, workloads as W

    if a.ensemble:
        ens = binding.Ensemble(W.ensemble_members(a.ensemble), config=dict(packing=0, ctas_per_sm=0, tile_policy=1))
        ens.step(a.warmup)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(ens.stream)
        ens.step(a.steps)
        ev1.record(ens.stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / max(a.steps, 1)
        print(json.dumps({"ensemble": a.ensemble, "ms_per_step": ms, "mlups": ens.nodes() / ms / 1e3,
                          "launches": ens.launches()}))
        ens.close()
        return

    wall = tuple(int(c in a.walls) for c in "xyz")
    p = W.params(lx=a.lx, ly=a.ly, lz=a.lz, wall=wall, kT=a.kT, radius=a.radius, g=a.g, G=a.G,
                 delta_rho=a.delta_rho)
    sim = binding.Sim(p)
    if a.adjoint:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(sim.stream)
        r = sim.adjoint(a.adjoint, a.checkpoint_every)
        ev1.record(sim.stream)
        torch.cuda.synchronize()
        print(json.dumps({"adjoint_steps": a.adjoint, "checkpoint_every": a.checkpoint_every,
                          "ms_per_step": ev0.elapsed_time(ev1) / a.adjoint, **r}))
        sim.close()
        return
    sim.step(a.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    kms = sim.step_timed(a.steps)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n = a.lx * a.ly * a.lz
    obs = sim.observables()
    print(json.dumps({"config": {k: getattr(a, k) for k in ("lx", "ly", "lz", "kT", "radius", "walls")},
                      "mlups": n * a.steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / a.steps,
                      "kernel_ms_per_step": {k: v / a.steps for k, v in kms.items()},
                      "launches": sim.launches(), "nonfinite": obs["nonfinite"]}))
    sim.close()


if __name__ == "__main__":
    main()
