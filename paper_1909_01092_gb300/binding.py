"""Thin ctypes binding of the C-ABI in include/flbm.h (argument marshalling only).

Every step of the method runs in the sm_103a kernels of libflbm. There is no
CPU path: if the shared library is missing or cannot be loaded, `load()`
raises. PyTorch provides the device memory of the populations (borrowed by
the library) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_LIB = None
_LOCK = threading.Lock()

# Every function declared in include/flbm.h.
EXPORTS = (
    "flbm_state_bytes", "flbm_create", "flbm_step", "flbm_particle_state", "flbm_observables",
    "flbm_read_fields", "flbm_write_fields", "flbm_set_particle", "flbm_run_host",
    "flbm_last_launch_count", "flbm_destroy", "flbm_error_string", "flbm_last_error",
    "flbm_step_timed", "flbm_kernel_name", "flbm_observables_noalloc",
    "flbm_checkpoint", "flbm_restore", "flbm_use_graphs", "flbm_use_tma", "flbm_set_tma_wait", "flbm_adjoint_run",
    "flbm_adjoint_tape_limit",
    "flbm_set_density_mode", "flbm_get_density_mode",
    "flbm_ensemble_create", "flbm_ensemble_step", "flbm_ensemble_tune", "flbm_ensemble_config",
    "flbm_ensemble_particles", "flbm_ensemble_read_fields", "flbm_ensemble_observables", "flbm_ensemble_nodes",
    "flbm_ensemble_last_launch_count", "flbm_ensemble_last_error", "flbm_ensemble_destroy",
)
NKERNELS = 4


class AdjResult(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("dJ_dg", ctypes.c_double), ("dJ_ddelta_rho", ctypes.c_double),
                ("dJ_dG", ctypes.c_double), ("steps", ctypes.c_int64), ("checkpoint_every", ctypes.c_int32),
                ("whole_tape", ctypes.c_int32), ("device_bytes", ctypes.c_double), ("ms_forward", ctypes.c_double),
                ("ms_reverse", ctypes.c_double)]


class EnsConfig(ctypes.Structure):
    _fields_ = [("packing", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("tile_policy", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("lz", ctypes.c_int32),
        ("wall_x", ctypes.c_int32), ("wall_y", ctypes.c_int32), ("wall_z", ctypes.c_int32),
        ("tau_s", ctypes.c_double), ("tau_d", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("G", ctypes.c_double), ("rho_a0", ctypes.c_double), ("rho_b0", ctypes.c_double),
        ("init_pert", ctypes.c_double), ("kT", ctypes.c_double), ("radius", ctypes.c_double),
        ("rho_p_ratio", ctypes.c_double), ("g", ctypes.c_double), ("delta_rho", ctypes.c_double),
        ("fluid_force", ctypes.c_double * 3), ("fluid_counterforce", ctypes.c_int32),
        ("replica", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("pos0", ctypes.c_double * 3),
    ]


class Particle(ctypes.Structure):
    _fields_ = [
        ("X", ctypes.c_double * 3), ("V", ctypes.c_double * 3), ("Vavg", ctypes.c_double * 3),
        ("Omega", ctypes.c_double * 3), ("F", ctypes.c_double * 3), ("T", ctypes.c_double * 3),
        ("P_pending", ctypes.c_double * 3), ("L_pending", ctypes.c_double * 3),
        ("delta", ctypes.c_double * 2), ("mp", ctypes.c_double), ("Fp", ctypes.c_double),
        ("nfluid", ctypes.c_int64), ("step", ctypes.c_int64),
    ]


class Obs(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double * 2), ("momentum", ctypes.c_double * 3), ("kinetic", ctypes.c_double),
        ("particle_momentum", ctypes.c_double * 3), ("pending_mass", ctypes.c_double * 2),
        ("nfluid", ctypes.c_int64), ("step", ctypes.c_int64), ("nonfinite", ctypes.c_int64),
        ("mode_temp", (ctypes.c_double * 19) * 2), ("diff_temp", ctypes.c_double * 3),
        ("mom_temp", ctypes.c_double * 3), ("n_bulk", ctypes.c_int64),
    ]


class FLBMError(RuntimeError):
    pass


def load(build_if_missing: bool = True):
    """Load libflbm (building it with nvcc if needed). Raises if unavailable."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.lib_path()
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise FLBMError(f"libflbm not built at {path}; run paper_1909_01092_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.flbm_state_bytes.restype = ctypes.c_size_t
        lib.flbm_state_bytes.argtypes = [ctypes.POINTER(Params)]
        lib.flbm_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        lib.flbm_step.argtypes = [vp, ctypes.c_int64]
        lib.flbm_particle_state.argtypes = [vp, ctypes.POINTER(Particle)]
        lib.flbm_observables.argtypes = [vp, ctypes.POINTER(Obs)]
        lib.flbm_read_fields.argtypes = [vp, fp, fp]
        lib.flbm_write_fields.argtypes = [vp, fp]
        lib.flbm_set_particle.argtypes = [vp, dp, dp, dp]
        lib.flbm_run_host.argtypes = [vp, fp, ctypes.c_int64, fp, ctypes.POINTER(Particle)]
        lib.flbm_step_timed.argtypes = [vp, ctypes.c_int64, dp]
        lib.flbm_observables_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, vp]
        lib.flbm_checkpoint.argtypes = [vp, ctypes.c_char_p]
        lib.flbm_restore.argtypes = [vp, ctypes.c_char_p]
        lib.flbm_use_graphs.argtypes = [vp, ctypes.c_int]
        lib.flbm_use_tma.argtypes = [vp, ctypes.c_int]
        lib.flbm_set_tma_wait.argtypes = [vp, ctypes.c_int64]
        lib.flbm_set_density_mode.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        lib.flbm_get_density_mode.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.flbm_adjoint_run.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(AdjResult)]
        lib.flbm_adjoint_tape_limit.argtypes = [vp, ctypes.c_int64]
        ens_p = ctypes.POINTER(EnsConfig)
        lib.flbm_ensemble_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, ens_p, vp,
                                             ctypes.POINTER(vp)]
        lib.flbm_ensemble_step.argtypes = [vp, ctypes.c_int64]
        lib.flbm_ensemble_tune.argtypes = [vp, ctypes.c_int32, ens_p, dp]
        lib.flbm_ensemble_config.argtypes = [vp, ens_p]
        lib.flbm_ensemble_particles.argtypes = [vp, ctypes.POINTER(Particle)]
        lib.flbm_ensemble_read_fields.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
        lib.flbm_ensemble_observables.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(Obs)]
        lib.flbm_ensemble_nodes.restype = ctypes.c_int64
        lib.flbm_ensemble_nodes.argtypes = [vp]
        lib.flbm_ensemble_last_launch_count.restype = ctypes.c_int64
        lib.flbm_ensemble_last_launch_count.argtypes = [vp]
        lib.flbm_ensemble_last_error.restype = ctypes.c_char_p
        lib.flbm_ensemble_last_error.argtypes = [vp]
        lib.flbm_ensemble_destroy.argtypes = [vp]
        lib.flbm_kernel_name.restype = ctypes.c_char_p
        lib.flbm_kernel_name.argtypes = [ctypes.c_int]
        lib.flbm_last_launch_count.restype = ctypes.c_int64
        lib.flbm_last_launch_count.argtypes = [vp]
        lib.flbm_destroy.argtypes = [vp]
        lib.flbm_error_string.restype = ctypes.c_char_p
        lib.flbm_error_string.argtypes = [ctypes.c_int]
        lib.flbm_last_error.restype = ctypes.c_char_p
        lib.flbm_last_error.argtypes = [vp]
        _LIB = lib
        return lib


def to_params(p: dict) -> Params:
    s = Params()
    s.lx, s.ly, s.lz = int(p["lx"]), int(p["ly"]), int(p["lz"])
    s.wall_x, s.wall_y, s.wall_z = (int(v) for v in p["wall"])
    s.tau_s, s.tau_d, s.tau_g = float(p["tau_s"]), float(p["tau_d"]), float(p["tau_g"])
    s.G = float(p["G"])
    s.rho_a0, s.rho_b0 = float(p["rho_a0"]), float(p["rho_b0"])
    s.init_pert, s.kT = float(p["init_pert"]), float(p["kT"])
    s.radius, s.rho_p_ratio = float(p["radius"]), float(p["rho_p_ratio"])
    s.g, s.delta_rho = float(p["g"]), float(p["delta_rho"])
    for a in range(3):
        s.fluid_force[a] = float(p["fluid_force"][a])
        s.pos0[a] = float(p["pos0"][a])
    s.fluid_counterforce = int(p["fluid_counterforce"])
    s.replica = int(p["replica"]) & 0xFFFFFFFF
    s.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    return s


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def record_bytes() -> int:
    return ctypes.sizeof(Particle)


def particle_dict(r: Particle) -> dict:
    d = {k: np.array(getattr(r, k)[:]) for k in ("X", "V", "Vavg", "Omega", "F", "T", "P_pending", "L_pending",
                                                  "delta")}
    d.update(mp=r.mp, Fp=r.Fp, nfluid=r.nfluid, step=r.step)
    return d


def obs_dict(r: Obs) -> dict:
    return dict(mass=np.array(r.mass[:]), momentum=np.array(r.momentum[:]), kinetic=r.kinetic,
                particle_momentum=np.array(r.particle_momentum[:]), pending_mass=np.array(r.pending_mass[:]),
                nfluid=r.nfluid, step=r.step, nonfinite=r.nonfinite,
                mode_temp=np.array([r.mode_temp[l][:] for l in range(2)]), diff_temp=np.array(r.diff_temp[:]),
                mom_temp=np.array(r.mom_temp[:]), n_bulk=r.n_bulk)


class Sim:
    """One simulation on the current CUDA device.

    The population storage (two float32 copies) is a torch CUDA tensor lent to
    the library; work is issued on torch's current stream unless `stream` (a
    torch.cuda.Stream) is given.
    """

    def __init__(self, p: dict, stream=None, borrow_torch: bool = True):
        import torch

        self.lib = load()
        self.p = dict(p)
        self._s = to_params(p)
        self.shape = (2, 19, p["lz"], p["ly"], p["lx"])
        self.N = p["lx"] * p["ly"] * p["lz"]
        nbytes = self.lib.flbm_state_bytes(ctypes.byref(self._s))
        if nbytes == 0:
            raise FLBMError("invalid parameters")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._buf = None
        ptr = None
        if borrow_torch:
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            ptr = ctypes.c_void_p(self._buf.data_ptr())
        h = ctypes.c_void_p()
        rc = self.lib.flbm_create(ctypes.byref(self._s), ptr, ctypes.c_size_t(nbytes),
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise FLBMError(f"flbm_create: {self.lib.flbm_error_string(rc).decode()}")
        self.h = h

    def _check(self, rc: int, what: str) -> None:
        if rc != 0:
            msg = self.lib.flbm_last_error(self.h).decode()
            raise FLBMError(f"{what}: {self.lib.flbm_error_string(rc).decode()} {msg}")

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.flbm_destroy(self.h)
            self.h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        self._check(self.lib.flbm_step(self.h, int(n)), "flbm_step")

    def adjoint(self, steps: int, checkpoint_every: int = 100, tape_limit: int | None = None) -> dict:
        """J = time-averaged settling velocity over the next `steps` steps and
        its gradient (dJ/dg, dJ/d delta_rho, dJ/dG) by the discrete adjoint;
        the simulation advances `steps` steps. `tape_limit` (bytes; None
        keeps the handle's setting, default automatic) bounds the tape of
        every step that spares the segment recomputes; 0 forces
        checkpoint-recompute."""
        if tape_limit is not None:
            self._check(self.lib.flbm_adjoint_tape_limit(self.h, int(tape_limit)), "flbm_adjoint_tape_limit")
        r = AdjResult()
        self._check(self.lib.flbm_adjoint_run(self.h, int(steps), int(checkpoint_every), ctypes.byref(r)),
                    "flbm_adjoint_run")
        d = {k: getattr(r, k) for k, _ in AdjResult._fields_}
        d["whole_tape"] = bool(d["whole_tape"])
        return d

    def use_graphs(self, enable: bool = True) -> None:
        """Replay flbm_step as captured eight-step CUDA graphs (needs a
        non-default stream)."""
        self._check(self.lib.flbm_use_graphs(self.h, int(bool(enable))), "flbm_use_graphs")

    def use_tma(self, enable: bool = True) -> None:
        """Select the bulk collide kernel with TMA-staged inputs (where the
        lattice allows it) or the one reading global memory directly (default)."""
        self._check(self.lib.flbm_use_tma(self.h, int(bool(enable))), "flbm_use_tma")

    def set_tma_wait(self, cycles: int) -> None:
        """Limit of the TMA-staged collide's waits for its tensor copies, in SM
        cycles (0: the default); a limit near 0 exercises the timeout path."""
        self._check(self.lib.flbm_set_tma_wait(self.h, int(cycles)), "flbm_set_tma_wait")

    def set_density_mode(self, mode: int, planes_per_block: int = 0) -> None:
        """0: density pass every step; 1: densities summed by the collide
        (fused), planes_per_block z-planes per block (0: automatic)."""
        self._check(self.lib.flbm_set_density_mode(self.h, int(mode), int(planes_per_block)),
                    "flbm_set_density_mode")

    def density_mode(self) -> tuple:
        """(mode, planes per block) the next step takes."""
        m, k = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.flbm_get_density_mode(self.h, ctypes.byref(m), ctypes.byref(k)), "flbm_get_density_mode")
        return m.value, k.value

    def checkpoint(self, path) -> None:
        self._check(self.lib.flbm_checkpoint(self.h, os.fsencode(path)), "flbm_checkpoint")

    def restore(self, path) -> None:
        self._check(self.lib.flbm_restore(self.h, os.fsencode(path)), "flbm_restore")

    def step_timed(self, n: int) -> dict:
        """Advance n steps; return the summed device milliseconds per kernel class."""
        ms = np.zeros(NKERNELS)
        self._check(self.lib.flbm_step_timed(self.h, int(n), _dptr(ms)), "flbm_step_timed")
        return {self.lib.flbm_kernel_name(k).decode(): float(ms[k]) for k in range(NKERNELS)}

    def launches(self) -> int:
        return int(self.lib.flbm_last_launch_count(self.h))

    def particle(self) -> dict:
        r = Particle()
        self._check(self.lib.flbm_particle_state(self.h, ctypes.byref(r)), "flbm_particle_state")
        return particle_dict(r)

    def observables(self, allow_nonfinite: bool = False) -> dict:
        r = Obs()
        rc = self.lib.flbm_observables(self.h, ctypes.byref(r))
        if not (allow_nonfinite and rc == -4):
            self._check(rc, "flbm_observables")
        return obs_dict(r)

    def read_f(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float32)
        self._check(self.lib.flbm_read_fields(self.h, _fptr(out), None), "flbm_read_fields")
        return out

    def read_rho(self) -> np.ndarray:
        out = np.empty((2,) + self.shape[2:], dtype=np.float32)
        self._check(self.lib.flbm_read_fields(self.h, None, _fptr(out)), "flbm_read_fields")
        return out

    def write_f(self, f: np.ndarray) -> None:
        a = np.ascontiguousarray(f, dtype=np.float32).reshape(self.shape)
        self._check(self.lib.flbm_write_fields(self.h, _fptr(a)), "flbm_write_fields")

    def set_particle(self, X, V=(0.0, 0.0, 0.0), Omega=(0.0, 0.0, 0.0)) -> None:
        x = np.asarray(X, dtype=np.float64)
        v = np.asarray(V, dtype=np.float64)
        w = np.asarray(Omega, dtype=np.float64)
        self._check(self.lib.flbm_set_particle(self.h, _dptr(x), _dptr(v), _dptr(w)), "flbm_set_particle")

    def run_host(self, f_in: np.ndarray, nsteps: int, f_out: np.ndarray | None = None, traj: bool = False):
        """End-to-end call: host populations in, nsteps, host populations (and the
        per-step particle records) out. `f_in`/`f_out` may be pinned torch tensors'
        numpy views."""
        a = np.ascontiguousarray(f_in, dtype=np.float32)
        tr = (Particle * max(int(nsteps), 1))() if traj else None
        self._check(self.lib.flbm_run_host(self.h, _fptr(a), int(nsteps),
                                           _fptr(f_out) if f_out is not None else None,
                                           tr if traj else None), "flbm_run_host")
        if traj:
            return [particle_dict(tr[k]) for k in range(int(nsteps))]
        return None


class Ensemble:
    """Many independent simulations advanced by batched launches.

    `plist` is a list of parameter dictionaries (one per replica). `config`
    is None (library default) or a dict with keys packing, ctas_per_sm,
    tile_policy. Work is issued on `stream` (a torch.cuda.Stream; default a
    new one, so that steps replay as CUDA graphs).
    """

    def __init__(self, plist, config=None, stream=None):
        import torch

        self.lib = load()
        self.plist = [dict(p) for p in plist]
        n = len(self.plist)
        arr = (Params * n)(*[to_params(p) for p in self.plist])
        self._arr = arr
        self.stream = stream if stream is not None else torch.cuda.Stream()
        cfg = None
        if config is not None:
            cfg = ctypes.byref(EnsConfig(int(config["packing"]), int(config["ctas_per_sm"]),
                                         int(config["tile_policy"])))
        h = ctypes.c_void_p()
        rc = self.lib.flbm_ensemble_create(arr, n, cfg, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise FLBMError(f"flbm_ensemble_create: {self.lib.flbm_error_string(rc).decode()}")
        self.h = h
        self.n = n

    def _check(self, rc: int, what: str) -> None:
        if rc != 0:
            msg = self.lib.flbm_ensemble_last_error(self.h).decode()
            raise FLBMError(f"{what}: {self.lib.flbm_error_string(rc).decode()} {msg}")

    def step(self, n: int = 1) -> None:
        self._check(self.lib.flbm_ensemble_step(self.h, int(n)), "flbm_ensemble_step")

    def tune(self, steps: int = 6):
        """Run the autotuner; return (chosen config dict, ms per step)."""
        c = EnsConfig()
        ms = np.zeros(1)
        self._check(self.lib.flbm_ensemble_tune(self.h, int(steps), ctypes.byref(c), _dptr(ms)), "flbm_ensemble_tune")
        return {"packing": c.packing, "ctas_per_sm": c.ctas_per_sm, "tile_policy": c.tile_policy}, float(ms[0])

    def config(self) -> dict:
        c = EnsConfig()
        self._check(self.lib.flbm_ensemble_config(self.h, ctypes.byref(c)), "flbm_ensemble_config")
        return {"packing": c.packing, "ctas_per_sm": c.ctas_per_sm, "tile_policy": c.tile_policy}

    def particles(self) -> list:
        recs = (Particle * self.n)()
        self._check(self.lib.flbm_ensemble_particles(self.h, recs), "flbm_ensemble_particles")
        return [particle_dict(r) for r in recs]

    def read_f(self, r: int) -> np.ndarray:
        p = self.plist[r]
        out = np.empty((2, 19, p["lz"], p["ly"], p["lx"]), dtype=np.float32)
        self._check(self.lib.flbm_ensemble_read_fields(self.h, int(r), _fptr(out)), "flbm_ensemble_read_fields")
        return out

    def observables(self, r: int) -> dict:
        o = Obs()
        rc = self.lib.flbm_ensemble_observables(self.h, int(r), ctypes.byref(o))
        if rc not in (0, -4):
            self._check(rc, "flbm_ensemble_observables")
        return obs_dict(o)

    def nodes(self) -> int:
        return int(self.lib.flbm_ensemble_nodes(self.h))

    def launches(self) -> int:
        return int(self.lib.flbm_ensemble_last_launch_count(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.flbm_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def settling_velocity(p: dict, steps: int, checkpoint_every: int = 100, v0=None):
    """torch.autograd.Function factory: returns f(g, delta_rho, G) -> J, the
    time-averaged settling velocity of `steps` noise-free steps of workload
    `p` (started at rest, or with particle velocity v0), whose backward pass
    is the hand-written adjoint of the step (flbm_adjoint_run)."""
    import torch

    class _SettlingVelocity(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g, delta_rho, G):
            q = dict(p, g=float(g), delta_rho=float(delta_rho), G=float(G))
            sim = Sim(q)
            if v0 is not None:
                sim.set_particle(q["pos0"], v0, (0.0, 0.0, 0.0))
            r = sim.adjoint(steps, checkpoint_every)
            sim.close()
            ctx.save_for_backward(torch.tensor([r["dJ_dg"], r["dJ_ddelta_rho"], r["dJ_dG"]], dtype=torch.float64))
            return torch.tensor(r["J"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            (gr,) = ctx.saved_tensors
            return gout * gr[0], gout * gr[1], gout * gr[2]

    return _SettlingVelocity.apply
