"""Seeded, synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds parameter sets and random-field generators only. It contains
none of the method's arithmetic, so both the CUDA path and the CPU oracle can
take their inputs from it without sharing any computation.

Parameter sets follow the paper's set-up (Section 3, "Numerical set-up and
Validation"): a square channel L x L with walls, a spherical particle at the
centre of the cross-section, driven along z by the force of Eq. (fp); the
fluid is a two-component Shan-Chen mixture (Section 2) with thermal noise of
strength kT.
"""
from __future__ import annotations

import copy

import numpy as np

# Keys every parameter dictionary carries (the C-ABI struct and the oracle's
# struct are filled from these).
KEYS = (
    "lx", "ly", "lz", "wall", "tau_s", "tau_d", "tau_g", "G", "rho_a0", "rho_b0",
    "init_pert", "kT", "radius", "rho_p_ratio", "g", "delta_rho", "fluid_force",
    "fluid_counterforce", "pos0", "seed", "replica",
)


def params(**over) -> dict:
    """A complete parameter dictionary: the defaults below, then `over`.

    Defaults: the noise-free channel of the small validation case (walls on x
    and y, periodic z), tau = 1 on every mode, G = 1.2, rho_A = 1.0,
    rho_B = 0.05, 1e-3 uniform perturbation, no particle. `pos0=None` places
    the particle at the centre ((lx-1)/2, (ly-1)/2, (lz-1)/2).
    """
    p = dict(
        lx=16, ly=16, lz=32, wall=(1, 1, 0),
        tau_s=1.0, tau_d=1.0, tau_g=1.0,
        G=1.2, rho_a0=1.0, rho_b0=0.05, init_pert=1e-3,
        kT=0.0, radius=0.0, rho_p_ratio=1.5, g=0.0, delta_rho=0.0,
        fluid_force=(0.0, 0.0, 0.0), fluid_counterforce=0,
        pos0=None, seed=1234, replica=0,
    )
    for k, v in over.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    if p["pos0"] is None:
        p["pos0"] = ((p["lx"] - 1) / 2.0, (p["ly"] - 1) / 2.0, (p["lz"] - 1) / 2.0)
    p["wall"] = tuple(int(w) for w in p["wall"])
    p["fluid_force"] = tuple(float(v) for v in p["fluid_force"])
    p["pos0"] = tuple(float(v) for v in p["pos0"])
    return p


# ---------------------------------------------------------------------------
# The workloads: a 16x16x32 noise-free channel with a sphere of radius 3; a
# 32x32x64 fluctuating channel with radius 4; a batched ensemble of uneven
# channels; a 128x128x512 fluctuating channel with radius 12 for the
# throughput roofline; a 64x64x128 noise-free channel for gradients.
# ---------------------------------------------------------------------------
def channel_small(**over) -> dict:
    """16x16x32 channel, walls on x and y, noise-free, sphere R=3, rho_p = 1.5 rho,
    body force 1e-5 along z, wetting 0; the case the oracle runs in seconds."""
    base = dict(lx=16, ly=16, lz=32, radius=3.0, rho_p_ratio=1.5, g=1e-5, kT=0.0, delta_rho=0.0)
    base.update(over)
    return params(**base)


def channel_fluct(delta_rho: float = 0.0, **over) -> dict:
    """32x32x64 channel with kT = 1e-5, sphere R=4, body force 5e-6 along z."""
    base = dict(lx=32, ly=32, lz=64, radius=4.0, rho_p_ratio=1.5, g=5e-6, kT=1e-5, delta_rho=delta_rho)
    base.update(over)
    return params(**base)


def channel_large(**over) -> dict:
    """128x128x512 channel with kT = 1e-5, sphere R=12, body force 1e-5 along z:
    the throughput workload (2 x 19 x 8.4M FP32 populations per copy)."""
    base = dict(lx=128, ly=128, lz=512, radius=12.0, rho_p_ratio=1.5, g=1e-5, kT=1e-5, delta_rho=0.0)
    base.update(over)
    return params(**base)


def channel_adjoint(**over) -> dict:
    """64x64x128 noise-free channel, sphere R=8, G=1.2, wetting 0.3, body force 1e-5."""
    base = dict(lx=64, ly=64, lz=128, radius=8.0, rho_p_ratio=1.5, g=1e-5, kT=0.0, delta_rho=0.3)
    base.update(over)
    return params(**base)


def ensemble_members(n: int = 128, seed: int = 1234) -> list[dict]:
    """Replicas of uneven size: L in {16,24,32,48} (length 2L), R in {2.5,4,6},
    kT in {1e-6,1e-5,1e-4}, assigned round-robin over the 36 combinations, body
    force log-uniform in [1e-6, 1e-5] from the seed, Philox replica index r."""
    rng = np.random.default_rng(seed)
    combos = [(L, R, kT) for L in (16, 24, 32, 48) for R in (2.5, 4.0, 6.0) for kT in (1e-6, 1e-5, 1e-4)]
    out = []
    for r in range(n):
        L, R, kT = combos[r % len(combos)]
        g = float(10.0 ** rng.uniform(-6.0, -5.0))
        out.append(params(lx=L, ly=L, lz=2 * L, radius=R, kT=kT, g=g, seed=seed, replica=r))
    return out


def random_populations(p: dict, seed: int, amp: float = 0.05, vel: float = 0.02) -> np.ndarray:
    """A seeded non-equilibrium population field, shape (2, 19, lz, ly, lx), float64.

    Each node gets the lattice-weight profile scaled to the component's
    initial density, a random density factor in [1-amp, 1+amp], a random
    first-moment tilt of size `vel` and independent random noise of size
    amp/4 on every direction (so every mode of the collision is exercised).
    Only random numbers and the printed D3Q19 weights are used.
    """
    rng = np.random.default_rng(seed)
    lx, ly, lz = p["lx"], p["ly"], p["lz"]
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    cz = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1], dtype=float)
    cx = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0], dtype=float)
    cy = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1], dtype=float)
    out = np.empty((2, 19, lz, ly, lx))
    for l, r0 in enumerate((p["rho_a0"], p["rho_b0"])):
        dens = r0 * (1.0 + amp * rng.uniform(-1, 1, size=(lz, ly, lx)))
        tilt = vel * rng.uniform(-1, 1, size=(3, lz, ly, lx))
        shape = (1.0 + 3.0 * (cx[:, None, None, None] * tilt[0] + cy[:, None, None, None] * tilt[1]
                              + cz[:, None, None, None] * tilt[2]))
        noise = 1.0 + 0.25 * amp * rng.uniform(-1, 1, size=(19, lz, ly, lx))
        out[l] = w[:, None, None, None] * dens[None] * shape * noise
    return out


def layered_populations(p: dict, rho_major: float = 2.21, rho_minor: float = 0.09, axis: int = 2,
                        lo: int | None = None, hi: int | None = None) -> np.ndarray:
    """Two-phase initial state, shape (2, 19, lz, ly, lx), float64: nodes with
    lo <= coordinate < hi along `axis` hold rho_A = rho_major, rho_B =
    rho_minor, the rest the opposite, each at rest (w_i rho_l). Defaults: the
    middle half of the axis. The densities default to the bulk values the
    paper prints for G = 1.5."""
    L = (p["lx"], p["ly"], p["lz"])[axis]
    lo = L // 4 if lo is None else lo
    hi = 3 * L // 4 if hi is None else hi
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    coord = np.indices((p["lz"], p["ly"], p["lx"]))[2 - axis]
    inside = (coord >= lo) & (coord < hi)
    rA = np.where(inside, rho_major, rho_minor)
    rB = np.where(inside, rho_minor, rho_major)
    return np.stack([w[:, None, None, None] * rA[None], w[:, None, None, None] * rB[None]])


def copy_params(p: dict) -> dict:
    return copy.deepcopy(p)
