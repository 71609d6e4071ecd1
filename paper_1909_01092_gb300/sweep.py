"""Settling statistics of the paper's Section 3 on the ensemble engine.

    python -m paper_1909_01092_gb300.sweep --L 16 24 32 48 --radius 3 --kT 1e-4 --g 2e-4

runs one ensemble of channels (L x L x 2L, walls on x and y, the fluid
counterforce so that the total external force vanishes) and prints one JSON
line per channel: the mean settling velocity U relative to the mean fluid
velocity, its velocity fluctuation Delta U, both with error bars, the
confinement ratio c_m = U / U_0 with U_0 = F_p / (3 pi eta d) (Eq. (cm)), and
the Langevin predictions Delta U^2 = kT / m_p (Eq. (FLUCTUATIONSSCALING)) and
Delta U / U (Eq. (normalizedconf)), confined and unconfined (c_m = 1).

Error bars follow the figure captions of Section 3: in the stationary state the
record is split into five equal time intervals, and the error is the standard
deviation of the interval values. The arithmetic here is host-side
post-processing of the particle records; every step runs in the CUDA kernels.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def interval_stats(v: np.ndarray, n: int = 5) -> dict:
    """Mean and fluctuation of a stationary series v (one particle velocity
    component, equally spaced samples), each with the standard deviation over
    n equal time intervals. The fluctuation of an interval is its standard
    deviation about its own mean."""
    v = np.asarray(v, dtype=np.float64)
    m = len(v) // n
    if m < 2:
        raise ValueError("need at least two samples per interval")
    blocks = v[: n * m].reshape(n, m)
    means = blocks.mean(axis=1)
    stds = blocks.std(axis=1)
    return {"mean": float(means.mean()), "mean_err": float(means.std()),
            "fluct": float(stds.mean()), "fluct_err": float(stds.std())}


def settling_row(p: dict, vz: np.ndarray, ufl: float, mp: float, Fp: float, intervals: int = 5) -> dict:
    """Statistics of one replica: p its parameters, vz its particle velocity
    record along z (equally spaced, stationary), ufl the mean fluid velocity
    along z, mp the particle mass and Fp the driving force (Eq. (fp)).

    U and Delta U are the interval mean and fluctuation of vz - ufl. The
    unconfined Stokes velocity is U_0 = F_p / (3 pi eta d), eta = rho_tot
    (tau_s - 1/2) / 3, so c_m = U / U_0 (Eq. (cm)). The Langevin predictions
    are Delta U = sqrt(kT / m_p) (Eq. (FLUCTUATIONSSCALING)) and
    Delta U / U = sqrt(kT / m_p) / (c_m U_0) (Eq. (normalizedconf)), whose
    unconfined form sets c_m = 1."""
    st = interval_stats(vz, intervals)
    eta = (p["rho_a0"] + p["rho_b0"]) * (p["tau_s"] - 0.5) / 3.0
    U = st["mean"] - ufl
    U0 = Fp / (3.0 * math.pi * eta * 2.0 * p["radius"])
    dU_pred = math.sqrt(p["kT"] / mp)
    return {"L": p["lx"], "d_over_L": 2.0 * p["radius"] / p["lx"], "kT": p["kT"], "g": p["g"],
            "U": U, "U_err": st["mean_err"], "dU": st["fluct"], "dU_err": st["fluct_err"],
            "cm": U / U0, "cm_err": st["mean_err"] / U0,
            "dU_pred": dU_pred, "dU_over_U": st["fluct"] / U, "dU_over_U_pred": dU_pred / U,
            "dU0_over_U0_pred": dU_pred / U0}


def settling_sweep(plist: list[dict], burn: int, samples: int, every: int = 10, intervals: int = 5) -> list[dict]:
    """Advance the replicas of plist as one ensemble: burn steps, then
    samples x every steps, recording Vavg_z every `every` steps. Returns one
    settling_row per replica. Needs the CUDA library (binding.Ensemble)."""
    from . import binding

    ens = binding.Ensemble(plist)
    try:
        ens.step(burn)
        rec = np.empty((samples, len(plist)))
        for k in range(samples):
            ens.step(every)
            rec[k] = [p["Vavg"][2] for p in ens.particles()]
        obs = [ens.observables(r) for r in range(len(plist))]
        parts = ens.particles()
    finally:
        ens.close()
    out = []
    for r, p in enumerate(plist):
        ufl = obs[r]["momentum"][2] / float(np.sum(obs[r]["mass"]))
        row = settling_row(p, rec[:, r], ufl, parts[r]["mp"], parts[r]["Fp"], intervals)
        row["nonfinite"] = int(obs[r]["nonfinite"])
        out.append(row)
    return out


def main(argv=None) -> None:
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[16, 24, 32, 48])
    ap.add_argument("--radius", type=float, default=3.0)
    ap.add_argument("--rho-p", type=float, default=5.0, help="particle density / fluid density")
    ap.add_argument("--kT", type=float, default=1e-4)
    ap.add_argument("--g", type=float, default=2e-4)
    ap.add_argument("--realisations", type=int, default=2)
    ap.add_argument("--burn", type=int, default=10000)
    ap.add_argument("--samples", type=int, default=1500)
    ap.add_argument("--every", type=int, default=10)
    a = ap.parse_args(argv)
    plist = [W.params(lx=L, ly=L, lz=2 * L, radius=a.radius, rho_p_ratio=a.rho_p, g=a.g, kT=a.kT, init_pert=0.0,
                      fluid_counterforce=1, replica=a.realisations * k + s)
             for k, L in enumerate(a.L) for s in range(a.realisations)]
    for row in settling_sweep(plist, a.burn, a.samples, a.every):
        print(json.dumps(row))


if __name__ == "__main__":
    main()
