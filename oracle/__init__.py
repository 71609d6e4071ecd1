"""ctypes binding of the FP64 CPU oracle (flbm_oracle.c).

TEST INFRASTRUCTURE. The oracle is the correctness reference for the GPU
library: a plain, slow FP64 implementation of the time step of the
fluctuating two-component Shan-Chen lattice Boltzmann method with a wetted
finite-size particle (arXiv:1909.01092, Section 2, Eqs. (density), (lbe),
(sc-force); Section 3, Eq. (fp)). Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it. It imports nothing from the GPU
package and shares no code with it; parameter dictionaries come from
`paper_1909_01092_gb300.workloads` (inputs only).

The shared object is compiled on first use with gcc (OpenMP if available)
into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def _lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, OpenMP when the compiler supports it)."""
    out = _lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


class _Params(ctypes.Structure):
    _fields_ = [
        ("lx", ctypes.c_int64), ("ly", ctypes.c_int64), ("lz", ctypes.c_int64),
        ("wall", ctypes.c_int64 * 3),
        ("tau_s", ctypes.c_double), ("tau_d", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("G", ctypes.c_double),
        ("rho0", ctypes.c_double * 2),
        ("init_pert", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("radius", ctypes.c_double), ("rho_p_ratio", ctypes.c_double),
        ("g", ctypes.c_double), ("delta_rho", ctypes.c_double),
        ("fluid_force", ctypes.c_double * 3),
        ("fluid_counterforce", ctypes.c_int64),
        ("pos0", ctypes.c_double * 3),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_int64),
    ]


def _load():
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [ctypes.POINTER(_Params)]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_step.argtypes = [P, ctypes.c_int64]
        lib.oracle_num_nodes.restype = ctypes.c_int64
        lib.oracle_num_nodes.argtypes = [P]
        lib.oracle_get_f.argtypes = [P, dp]
        lib.oracle_set_f.argtypes = [P, dp]
        lib.oracle_get_particle.argtypes = [P, dp]
        lib.oracle_set_particle.argtypes = [P, dp, dp, dp]
        lib.oracle_fields.argtypes = [P, dp, dp, dp, dp, dp]
        lib.oracle_observables.argtypes = [P, dp]
        lib.oracle_mode_temps.argtypes = [P, dp]
        lib.oracle_lattice.argtypes = [dp, dp, ctypes.POINTER(ctypes.c_int64), dp, dp]
        lib.oracle_philox.argtypes = [u32p, u32p, u32p]
        lib.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32, dp]
        lib.oracle_uniform.restype = ctypes.c_double
        lib.oracle_uniform.argtypes = [ctypes.c_uint32]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _LIB = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _to_struct(p: dict) -> _Params:
    s = _Params()
    s.lx, s.ly, s.lz = int(p["lx"]), int(p["ly"]), int(p["lz"])
    for a in range(3):
        s.wall[a] = int(p["wall"][a])
        s.fluid_force[a] = float(p["fluid_force"][a])
        s.pos0[a] = float(p["pos0"][a])
    s.tau_s, s.tau_d, s.tau_g = float(p["tau_s"]), float(p["tau_d"]), float(p["tau_g"])
    s.G = float(p["G"])
    s.rho0[0], s.rho0[1] = float(p["rho_a0"]), float(p["rho_b0"])
    s.init_pert = float(p["init_pert"])
    s.kT = float(p["kT"])
    s.radius = float(p["radius"])
    s.rho_p_ratio = float(p["rho_p_ratio"])
    s.g = float(p["g"])
    s.delta_rho = float(p["delta_rho"])
    s.fluid_counterforce = int(p["fluid_counterforce"])
    s.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    s.replica = int(p["replica"])
    return s


PARTICLE_FIELDS = ("X", "V", "Vavg", "Omega", "F", "T", "Ppend", "Lpend")


class Oracle:
    """One simulation held by the oracle. Populations are float64 arrays of
    shape (2, 19, lz, ly, lx): component A/B, D3Q19 direction, z, y, x."""

    def __init__(self, p: dict):
        self.lib = _load()
        self.p = dict(p)
        self._s = _to_struct(p)
        self.h = self.lib.oracle_create(ctypes.byref(self._s))
        if not self.h:
            raise MemoryError("oracle_create failed")
        self.shape = (2, 19, p["lz"], p["ly"], p["lx"])
        self.N = p["lx"] * p["ly"] * p["lz"]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_destroy(h)
            self.h = None

    def step(self, n: int = 1) -> None:
        self.lib.oracle_step(self.h, int(n))

    def get_f(self) -> np.ndarray:
        out = np.empty(self.shape)
        self.lib.oracle_get_f(self.h, _dptr(out))
        return out

    def set_f(self, f: np.ndarray) -> None:
        a = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape)
        self.lib.oracle_set_f(self.h, _dptr(a))

    def particle(self) -> dict:
        out = np.empty(32)
        self.lib.oracle_get_particle(self.h, _dptr(out))
        d = {k: out[3 * i:3 * i + 3].copy() for i, k in enumerate(PARTICLE_FIELDS)}
        d["delta"] = out[24:26].copy()
        d["nfluid"] = int(out[26])
        d["step"] = int(out[27])
        d["mp"] = float(out[28])
        d["Fp"] = float(out[29])
        return d

    def set_particle(self, X, V=(0, 0, 0), Omega=(0, 0, 0)) -> None:
        x = np.asarray(X, dtype=np.float64)
        v = np.asarray(V, dtype=np.float64)
        w = np.asarray(Omega, dtype=np.float64)
        self.lib.oracle_set_particle(self.h, _dptr(x), _dptr(v), _dptr(w))

    def fields(self) -> dict:
        n = self.N
        lz, ly, lx = self.shape[2:]
        rho = np.empty(2 * n)
        psi = np.empty(2 * n)
        force = np.empty(6 * n)
        solid = np.empty(n)
        fsc = np.empty(6)
        self.lib.oracle_fields(self.h, _dptr(rho), _dptr(psi), _dptr(force), _dptr(solid), _dptr(fsc))
        return dict(
            rho=rho.reshape(2, lz, ly, lx), psi=psi.reshape(2, lz, ly, lx),
            force=force.reshape(2, 3, lz, ly, lx), solid=solid.reshape(lz, ly, lx).astype(bool),
            sc_reaction_force=fsc[:3], sc_reaction_torque=fsc[3:],
        )

    def observables(self) -> dict:
        out = np.empty(11)
        self.lib.oracle_observables(self.h, _dptr(out))
        return dict(mass=out[0:2].copy(), momentum=out[2:5].copy(), kinetic=float(out[5]),
                    particle_momentum=out[6:9].copy(), pending_mass=out[9:11].copy())


    def mode_temps(self) -> dict:
        """Temperatures of the fluctuating modes over the bulk fluid nodes:
        mode_temp (2, 19) for k = 4..18, interdiffusion diff_temp (3),
        momentum mom_temp (3), node count n_bulk."""
        out = np.empty(45)
        self.lib.oracle_mode_temps(self.h, _dptr(out))
        return dict(mode_temp=out[:38].reshape(2, 19).copy(), diff_temp=out[38:41].copy(),
                    mom_temp=out[41:44].copy(), n_bulk=int(out[44]))


def lattice() -> dict:
    lib = _load()
    c = np.empty(57)
    w = np.empty(19)
    opp = np.empty(19, dtype=np.int64)
    e = np.empty(361)
    b = np.empty(19)
    lib.oracle_lattice(_dptr(c), _dptr(w), opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(e), _dptr(b))
    return dict(c=c.reshape(19, 3), w=w, opp=opp, e=e.reshape(19, 19), b=b)


def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_philox(c.ctypes.data_as(P), k.ctypes.data_as(P), o.ctypes.data_as(P))
    return o


def normals(seed: int, replica: int, step: int, node: int) -> np.ndarray:
    lib = _load()
    out = np.empty(36)
    lib.oracle_normals(int(seed) & 0xFFFFFFFFFFFFFFFF, int(replica), int(step) & 0xFFFFFFFF,
                       int(node) & 0xFFFFFFFF, _dptr(out))
    return out


def uniform(x: int) -> float:
    return _load().oracle_uniform(int(x) & 0xFFFFFFFF)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Thread count (n >= 1) for the OpenMP loops of the oracle's later calls."""
    _load().oracle_set_threads(int(n))
