"""Physics runs of the channel configurations and of Section 3's study, each
printing JSON (one object per run or per channel).

    python -m paper_1909_01092_gb300.physics settling       # 16x16x32 noise-free, 1000 steps
    python -m paper_1909_01092_gb300.physics fluctuating    # 32x32x64, kT=1e-5, three wettings
    python -m paper_1909_01092_gb300.physics confinement    # c_m and Delta U over d/L, three wettings
    python -m paper_1909_01092_gb300.physics production     # closed 60x60x900 channel timing

settling: the noise-free 16x16x32 channel (R = 3, rho_p = 1.5 rho, g = 1e-5
along z, walls on x and y): particle velocity and hydrodynamic force after
1000 steps, the settling velocity averaged over the last 200 steps, and
c_m = U / U_0 with U_0 = F_p / (3 pi eta d) (Section 3, Eq. (cm)).

fluctuating: the 32x32x64 channel at kT = 1e-5 (R = 4, g = 5e-6) for each
wetting parameter, as one ensemble (its members are the single simulations
bit for bit): mean settling velocity and the velocity variances along z and
across, each against kT / m_p (Section 3, Eq. (MEANVARIANCE)), with
five-interval error bars.

confinement: Section 3's sweep in the paper's fluid (G = 1.5, rho_A = 2.21,
rho_B = 0.09, tau = 1, rho_p = 2 rho_tot): channels of cross-section 60 x 60
with walls on x and y, periodic along z with the fluid counterforce (zero
net external force, as in the closed channel), d/L from 0.133 to 0.67 and
three wetting parameters, all replicas in one ensemble. Noise-free, it gives
c_m(d/L); with noise, Delta U against sqrt(kT / m_p) (Eq. (FLUCTUATIONSSCALING))
and Delta U / U against Eq. (normalizedconf), confined and unconfined.

production: the closed 60 x 60 x 900 channel of Section 3 (walls on every
axis, R = 8, the paper's fluid, kT = 1e-5, g = 5e-6): MLUPS of the fused and
two-pass steps.

Every step runs in the CUDA kernels; this module only sets up the runs and
reduces the particle records on the host.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import sweep

PAPER_FLUID = dict(G=1.5, rho_a0=2.21, rho_b0=0.09)


def _stokes(p: dict, Fp: float) -> float:
    """Unconfined Stokes velocity U_0 = F_p / (3 pi eta d), eta = rho_tot nu."""
    eta = (p["rho_a0"] + p["rho_b0"]) * (p["tau_s"] - 0.5) / 3.0
    return Fp / (3.0 * math.pi * eta * 2.0 * p["radius"])


def settling(steps: int = 1000, tail: int = 200) -> dict:
    import torch

    from . import binding, workloads as W

    p = W.channel_small()
    sim = binding.Sim(p, stream=torch.cuda.Stream())
    tr = sim.run_host(sim.read_f(), steps, traj=True)
    sim.close()
    vz = np.array([t["Vavg"][2] for t in tr])
    last = tr[-1]
    U = float(vz[-tail:].mean())
    U0 = _stokes(p, last["Fp"])
    return {"run": "settling", "workload": "channel_16x16x32_R3_noise_free", "steps": steps,
            "V": last["V"].tolist(), "Vavg": last["Vavg"].tolist(), "F": last["F"].tolist(), "Fp": last["Fp"],
            "mp": last["mp"], "U_last_200": U, "U0_stokes": U0, "cm": U / U0,
            "F_over_Fp": float(-last["F"][2] / last["Fp"]),
            "note": "velocities in lattice units per step; F is the hydrodynamic force of the last step"}


def fluctuating(steps: int = 200000, burn: int = 20000, every: int = 10, drhos=(-0.5, 0.0, 0.5)) -> list:
    import torch

    from . import binding, workloads as W

    plist = [W.channel_fluct(delta_rho=d) for d in drhos]
    ens = binding.Ensemble(plist, stream=torch.cuda.Stream())
    t0 = time.perf_counter()
    ens.step(burn)
    n = (steps - burn) // every
    V = np.empty((n, len(plist), 3))
    Va = np.empty((n, len(plist), 3))
    for k in range(n):
        ens.step(every)
        parts = ens.particles()
        V[k] = [q["V"] for q in parts]
        Va[k] = [q["Vavg"] for q in parts]
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    parts = ens.particles()
    ens.close()
    out = []
    for r, p in enumerate(plist):
        mp, Fp = parts[r]["mp"], parts[r]["Fp"]
        s_th = p["kT"] / mp
        row = {"run": "fluctuating", "workload": "channel_32x32x64_kT1e-5_R4", "delta_rho": p["delta_rho"],
               "steps": steps, "burn": burn, "sample_every": every, "seconds": secs, "kT_over_mp": s_th,
               "U0_stokes": _stokes(p, Fp)}
        for name, rec in (("V", V[:, r]), ("Vavg", Va[:, r])):
            z = sweep.interval_stats(rec[:, 2])
            x = sweep.interval_stats(rec[:, 0])
            y = sweep.interval_stats(rec[:, 1])
            row[name] = {"U": z["mean"], "U_err": z["mean_err"],
                         "var_z_over_kT_mp": z["fluct"] ** 2 / s_th,
                         "var_z_err": 2 * z["fluct"] * z["fluct_err"] / s_th,
                         "var_xy_over_kT_mp": 0.5 * (x["fluct"] ** 2 + y["fluct"] ** 2) / s_th,
                         "var_xy_err": (x["fluct"] * x["fluct_err"] + y["fluct"] * y["fluct_err"]) / s_th}
        row["cm"] = row["Vavg"]["U"] / row["U0_stokes"]
        out.append(row)
    return out


def confinement(L: int = 60, lz: int = 240, d_over_L=(0.133, 0.267, 0.4, 0.533, 0.667), drhos=(-0.1, 0.0, 0.1),
                kT: float = 0.0, g: float = 5e-5, burn: int = 20000, samples: int = 1000, every: int = 10) -> list:
    from . import workloads as W

    plist = []
    for dl in d_over_L:
        R = 0.5 * dl * L
        for d in drhos:
            plist.append(W.params(lx=L, ly=L, lz=lz, wall=(1, 1, 0), radius=R, rho_p_ratio=2.0, g=g, kT=kT,
                                  delta_rho=d, init_pert=0.0, fluid_counterforce=1, replica=len(plist),
                                  **PAPER_FLUID))
    t0 = time.perf_counter()
    rows = sweep.settling_sweep(plist, burn, samples, every)
    secs = time.perf_counter() - t0
    for row, p in zip(rows, plist):
        row.update(run="confinement", delta_rho=p["delta_rho"], lz=lz, burn=burn, samples=samples, every=every,
                   seconds_all_replicas=secs)
    return rows


def production(steps: int = 200, warmup: int = 10) -> list:
    import torch

    from . import binding, workloads as W

    p = W.params(lx=60, ly=60, lz=900, wall=(1, 1, 1), radius=8.0, rho_p_ratio=2.0, kT=1e-5, g=5e-6,
                 **PAPER_FLUID)
    out = []
    for mode in (1, 0):
        sim = binding.Sim(p, stream=torch.cuda.Stream())
        sim.set_density_mode(mode)
        sim.step(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        kms = sim.step_timed(steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n = p["lx"] * p["ly"] * p["lz"]
        out.append({"run": "production", "workload": "closed_channel_60x60x900_R8_kT1e-5", "density_mode": mode,
                    "planes_per_block": sim.density_mode()[1], "ms_per_step": ms, "mlups": n / (ms * 1e-3) / 1e6,
                    "kernel_ms_per_step": {k: v / steps for k, v in kms.items()},
                    "nonfinite": sim.observables()["nonfinite"]})
        sim.close()
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("run", choices=("settling", "fluctuating", "confinement", "production"))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--kT", type=float, default=0.0, help="confinement: thermal energy (0: noise-free c_m)")
    ap.add_argument("--g", type=float, default=5e-5, help="confinement: body-force density")
    ap.add_argument("--lz", type=int, default=240, help="confinement: channel length")
    ap.add_argument("--burn", type=int, default=20000)
    ap.add_argument("--samples", type=int, default=1000)
    ap.add_argument("--every", type=int, default=10)
    a = ap.parse_args(argv)
    if a.run == "settling":
        rows = [settling(a.steps or 1000)]
    elif a.run == "fluctuating":
        rows = fluctuating(a.steps or 200000, burn=a.burn, every=a.every)
    elif a.run == "confinement":
        rows = confinement(lz=a.lz, kT=a.kT, g=a.g, burn=a.burn, samples=a.samples, every=a.every)
    else:
        rows = production(a.steps or 200)
    for r in rows:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
