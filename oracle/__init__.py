"""ctypes front end of the FP64 CPU oracle (picmcc_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle exists to check the CUDA library.  Only
the tests, the smoke check and the CPU-baseline leg of the benchmark import
this module; the library itself never does, and this module imports nothing
from the library.

Every function here is argument marshalling; the arithmetic is in the C file,
which cites the passages of the paper each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "picmcc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NMOM, NRES = 16, 24
ELASTIC, EXCITATION, IONIZATION, ATTACHMENT = 0, 1, 2, 3
Q_E, M_ELEC, EPS_0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


PD = C.POINTER(C.c_double)
PF = C.POINTER(C.c_float)
PI64 = C.POINTER(C.c_int64)
PU64 = C.POINTER(C.c_uint64)
PU32 = C.POINTER(C.c_uint32)
PU8 = C.POINTER(C.c_uint8)
PINT = C.POINTER(C.c_int)


class Setup(C.Structure):
    _fields_ = [("n_proc", C.c_int), ("n_bins", C.c_int), ("eps", PD), ("nu", PD),
                ("nu_max", C.c_double), ("kind", PINT), ("threshold", PD), ("mass", PD),
                ("dt", C.c_double), ("seed", C.c_uint64), ("prec", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double),
                ("mask", PU8), ("Ex", PF), ("Ey", PF), ("Ez", PF), ("E0", C.c_double * 3),
                ("boundary", C.c_int), ("photo_prob", C.c_double), ("chi_a", C.c_double),
                ("chi_b", C.c_double), ("axi", C.c_int), ("Ex64", PD), ("Ey64", PD), ("Ez64", PD),
                ("dt_kick", C.c_double)]


class Parts(C.Structure):
    _fields_ = [("n", C.c_longlong), ("cap", C.c_longlong)] + \
               [(k, PD) for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "w")] + \
               [("id", PU64)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in ("n_start", "n_children", "n_end", "n_attached",
                                             "n_absorbed", "n_null", "n_clamped", "n_events", "n_photo")] + \
               [("n_coll", C.c_longlong * 16), ("w_ion", C.c_double), ("w_att", C.c_double),
                ("w_absorbed", C.c_double)]


class MSStats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in ("n_before", "n_after", "n_merged_pairs",
                                             "n_split_added", "n_cells")] + [("scale", C.c_double)]


class SwarmCfg(C.Structure):
    _fields_ = [("n0", C.c_longlong), ("n_lo", C.c_longlong), ("n_hi", C.c_longlong),
                ("n_steps", C.c_int), ("kT_eV", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_philox.argtypes = [PU32, PU32, PU32]
            L.orc_rate_table.argtypes = [C.c_int, C.c_int, PD, PD, PD, PD, PD]
            L.orc_rate_table.restype = C.c_int
            L.orc_step.argtypes = [C.POINTER(Setup), C.POINTER(Parts), C.c_uint32, C.c_int,
                                   PI64, PI64, PI64, C.POINTER(Stats)]
            L.orc_step.restype = C.c_int
            L.orc_deposit.argtypes = [C.POINTER(Setup), C.POINTER(Parts), PI64]
            L.orc_fixed_to_rho.argtypes = [C.c_longlong, C.c_double, PI64, PI64, PI64, PD]
            L.orc_seed_gaussian.argtypes = [C.POINTER(Setup), C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_double, C.c_double, C.c_uint64,
                                            C.POINTER(Parts)]
            L.orc_seed_gaussian.restype = C.c_longlong
            L.orc_seed_maxwell.argtypes = [C.POINTER(Setup), C.c_longlong, C.c_double,
                                           C.POINTER(Parts)]
            L.orc_merge_split.argtypes = [C.POINTER(Setup), C.POINTER(Parts), C.c_uint32, C.c_int,
                                          C.c_double, C.c_longlong, C.POINTER(MSStats)]
            L.orc_merge_split.restype = C.c_int
            L.orc_poisson_cg.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, PD, PU8, C.c_double,
                                         C.c_double, C.c_double, PD, C.c_double, C.c_int, PD, PINT]
            L.orc_poisson_cg.restype = C.c_int
            L.orc_grad_phi.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, PD, C.c_double,
                                       C.c_double, PD, PD, PD]
            L.orc_poisson_axi.argtypes = [C.c_int, C.c_int, C.c_double, PD, PU8, C.c_double, C.c_double,
                                          C.c_double, PD, C.c_double, C.c_int, PD, PINT]
            L.orc_poisson_axi.restype = C.c_int
            L.orc_grad_axi.argtypes = [C.c_int, C.c_int, C.c_double, PD, C.c_double, C.c_double, PD, PD]
            L.orc_fixed_to_rho_axi.argtypes = [C.c_int, C.c_int, C.c_double, PI64, PI64, PI64, PD]
            L.orc_swarm_run.argtypes = [C.POINTER(Setup), C.POINTER(SwarmCfg), C.POINTER(Parts), PD,
                                        C.POINTER(C.c_longlong)]
            L.orc_swarm_run.restype = C.c_int
            L.orc_swarm_coefficients.argtypes = [PD, C.c_int, C.c_int, C.c_double, C.c_double, PD]
            L.orc_swarm_coefficients.restype = C.c_int
            L.orc_gather_field.argtypes = [C.POINTER(Setup), C.c_longlong, PD, PD, PD, PD]
            L.orc_photon_draws.argtypes = [C.POINTER(Setup), C.c_uint64, C.c_uint32, C.c_int, PINT, PD, PD]
            L.orc_rates_at_energy.argtypes = [C.POINTER(Setup), C.c_longlong, PD, PD]
            L.orc_draw.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, PD]
            L.orc_derived_id.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
            L.orc_derived_id.restype = C.c_uint64
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


# ----------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c, PU32), _p(k, PU32), _p(o, PU32))
    return o


def draw(seed: int, pid: int, step: int, k: int) -> np.ndarray:
    u = np.zeros(4)
    lib().orc_draw(seed, pid, step, k, _p(u, PD))
    return u


def derived_id(seed: int, pid: int, step: int, tag: int) -> int:
    return int(lib().orc_derived_id(seed, pid, step, tag))


def rate_table(gas: dict):
    sig = np.ascontiguousarray(gas["sigma"], dtype=np.float64)
    n_proc, n_bins = sig.shape
    nu = np.zeros_like(sig)
    numax = C.c_double()
    eps = np.ascontiguousarray(gas["eps"], np.float64)
    dens = np.ascontiguousarray(gas["density"], np.float64)
    rc = lib().orc_rate_table(n_proc, n_bins, _p(eps, PD), _p(sig, PD), _p(dens, PD), _p(nu, PD),
                              C.byref(numax))
    if rc:
        raise ValueError("orc_rate_table failed")
    return nu, numax.value


class Model:
    """Holds an orc_setup and the arrays it points to."""

    def __init__(self, gas: dict, dt: float, seed: int, prec: int = 64, grid: dict | None = None,
                 field=None, E0=(0.0, 0.0, 0.0), mask=None, boundary: int = 0, photo=None, axi: bool = False,
                 dt_kick: float = 0.0):
        """photo: None, or dict(xi, pq, pressure, p_o2, chi_min, chi_max) (Pa and 1/(m Pa)).
        field: three [nz][ny][nx] arrays, float32 or float64 (all the same type).
        dt_kick: length of the half-kick completing the previous step's Eq. 2 (0 = dt)."""
        self.gas = gas
        self.nu, self.nu_max = rate_table(gas)
        self._keep = [np.ascontiguousarray(gas["eps"], np.float64), self.nu,
                      np.ascontiguousarray(gas["kind"], np.int32),
                      np.ascontiguousarray(gas["threshold"], np.float64),
                      np.ascontiguousarray(gas["mass"], np.float64)]
        s = Setup()
        s.n_proc, s.n_bins = self.nu.shape
        s.eps, s.nu = _p(self._keep[0], PD), _p(self.nu, PD)
        s.nu_max = self.nu_max
        s.kind, s.threshold, s.mass = _p(self._keep[2], PINT), _p(self._keep[3], PD), _p(self._keep[4], PD)
        s.dt, s.seed, s.prec = dt, seed, prec
        if grid is not None:
            s.nx, s.ny, s.nz, s.dx = grid["nx"], grid["ny"], grid["nz"], grid["dx"]
            s.ox, s.oy, s.oz = grid["origin"]
        if mask is not None:
            m = np.ascontiguousarray(mask, np.uint8)
            self._keep.append(m)
            s.mask = _p(m, PU8)
        if field is not None:
            if all(np.asarray(f).dtype == np.float64 for f in field):
                fs = [np.ascontiguousarray(f, np.float64) for f in field]
                self._keep += fs
                s.Ex64, s.Ey64, s.Ez64 = (_p(f, PD) for f in fs)
            else:
                fs = [np.ascontiguousarray(f, np.float32) for f in field]
                self._keep += fs
                s.Ex, s.Ey, s.Ez = (_p(f, PF) for f in fs)
        s.dt_kick = dt_kick
        s.E0[0], s.E0[1], s.E0[2] = E0
        s.boundary = boundary
        s.axi = int(axi)
        if photo is not None and photo["xi"] > 0:
            s.photo_prob = photo["xi"] * photo["pq"] / (photo["pressure"] + photo["pq"])
            s.chi_a = photo["chi_min"] * photo["p_o2"]
            s.chi_b = photo["chi_max"] * photo["p_o2"]
        self.s = s
        self.grid = grid

    @property
    def ncell(self):
        g = self.grid
        return g["nx"] * g["ny"] * g["nz"]


class Particles:
    """Growable-by-capacity SoA of float64 particles for the oracle."""
    F = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "w")

    def __init__(self, cap: int, init: dict | None = None):
        self.arr = {k: np.zeros(cap) for k in self.F}
        self.arr["id"] = np.zeros(cap, np.uint64)
        self.c = Parts()
        self.c.cap = cap
        for k in self.F:
            setattr(self.c, k, _p(self.arr[k], PD))
        self.c.id = _p(self.arr["id"], PU64)
        self.c.n = 0
        if init is not None:
            n = len(init["x"])
            assert n <= cap
            for k in self.F + ("id",):
                if k in init:
                    self.arr[k][:n] = init[k]
            self.c.n = n

    @property
    def n(self):
        return int(self.c.n)

    def view(self) -> dict:
        return {k: v[: self.n].copy() for k, v in self.arr.items()}


def step(m: Model, p: Particles, step_idx: int, first: bool, q_e=None, q_pos=None, q_neg=None):
    st = Stats()
    rc = lib().orc_step(C.byref(m.s), C.byref(p.c), step_idx, int(first), _p(q_e, PI64),
                        _p(q_pos, PI64), _p(q_neg, PI64), C.byref(st))
    return rc, st


def deposit(m: Model, p: Particles) -> np.ndarray:
    q = np.zeros(m.ncell, np.int64)
    lib().orc_deposit(C.byref(m.s), C.byref(p.c), _p(q, PI64))
    return q


def fixed_to_rho(dV: float, q_e, q_pos, q_neg) -> np.ndarray:
    q_e, q_pos, q_neg = (np.ascontiguousarray(a, np.int64) for a in (q_e, q_pos, q_neg))
    rho = np.zeros(q_e.size)
    lib().orc_fixed_to_rho(q_e.size, dV, _p(q_e, PI64), _p(q_pos, PI64), _p(q_neg, PI64), _p(rho, PD))
    return rho


def seed_gaussian(m: Model, n0, radius, center, w0, cap, id0=0) -> Particles:
    p = Particles(cap)
    n = lib().orc_seed_gaussian(C.byref(m.s), n0, radius, center[0], center[1], center[2], w0, id0,
                                C.byref(p.c))
    if n < 0:
        raise RuntimeError("capacity")
    return p


def merge_split(m: Model, p: Particles, step_idx: int, n_ppc: int = 75, w_min: float = 1.0,
                cap: int = 0):
    ms = MSStats()
    rc = lib().orc_merge_split(C.byref(m.s), C.byref(p.c), step_idx, n_ppc, w_min, cap, C.byref(ms))
    return rc, ms


def poisson(grid: dict, rho, mask, v_mask, v_lo, v_hi, rtol=1e-12, max_iter=100000, phi0=None):
    nx, ny, nz, h = grid["nx"], grid["ny"], grid["nz"], grid["dx"]
    rho = np.ascontiguousarray(rho, np.float64).ravel()
    phi = np.zeros(nx * ny * nz) if phi0 is None else np.ascontiguousarray(phi0, np.float64).ravel().copy()
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8).ravel()
    rr, it = C.c_double(), C.c_int()
    rc = lib().orc_poisson_cg(nx, ny, nz, h, _p(rho, PD), _p(mk, PU8), v_mask, v_lo, v_hi, _p(phi, PD),
                              rtol, max_iter, C.byref(rr), C.byref(it))
    if rc:
        raise RuntimeError("orc_poisson_cg failed")
    return phi.reshape(nz, ny, nx), rr.value, it.value


def grad_phi(grid: dict, phi, v_lo, v_hi):
    nx, ny, nz, h = grid["nx"], grid["ny"], grid["nz"], grid["dx"]
    phi = np.ascontiguousarray(phi, np.float64).ravel()
    E = [np.zeros(nx * ny * nz) for _ in range(3)]
    lib().orc_grad_phi(nx, ny, nz, h, _p(phi, PD), v_lo, v_hi, *(_p(e, PD) for e in E))
    return tuple(e.reshape(nz, ny, nx) for e in E)


def poisson_axi(nr: int, nz: int, h: float, rho, mask, v_mask, v_lo, v_hi, rtol=1e-12, max_iter=200000,
                phi0=None):
    """Axisymmetric solve on [nz][nr] ring cells; returns (phi, rel_res, iterations)."""
    rho = np.ascontiguousarray(rho, np.float64).ravel()
    phi = np.zeros(nr * nz) if phi0 is None else np.ascontiguousarray(phi0, np.float64).ravel().copy()
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8).ravel()
    rr, it = C.c_double(), C.c_int()
    rc = lib().orc_poisson_axi(nr, nz, h, _p(rho, PD), _p(mk, PU8), v_mask, v_lo, v_hi, _p(phi, PD), rtol,
                               max_iter, C.byref(rr), C.byref(it))
    if rc:
        raise RuntimeError("orc_poisson_axi failed")
    return phi.reshape(nz, nr), rr.value, it.value


def grad_axi(nr: int, nz: int, h: float, phi, v_lo, v_hi):
    phi = np.ascontiguousarray(phi, np.float64).ravel()
    Er, Ez = np.zeros(nr * nz), np.zeros(nr * nz)
    lib().orc_grad_axi(nr, nz, h, _p(phi, PD), v_lo, v_hi, _p(Er, PD), _p(Ez, PD))
    return Er.reshape(nz, nr), Ez.reshape(nz, nr)


def fixed_to_rho_axi(nr: int, nz: int, dx: float, q_e, q_pos, q_neg) -> np.ndarray:
    q_e, q_pos, q_neg = (np.ascontiguousarray(a, np.int64) for a in (q_e, q_pos, q_neg))
    rho = np.zeros(q_e.size)
    lib().orc_fixed_to_rho_axi(nr, nz, dx, _p(q_e, PI64), _p(q_pos, PI64), _p(q_neg, PI64), _p(rho, PD))
    return rho


def gather_field(m: Model, x, y, z) -> np.ndarray:
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    E = np.zeros((len(x), 3))
    lib().orc_gather_field(C.byref(m.s), len(x), _p(x, PD), _p(y, PD), _p(z, PD), _p(E, PD))
    return E


def rates_at(m: Model, energies) -> np.ndarray:
    e = np.ascontiguousarray(energies, np.float64)
    out = np.zeros((len(e), m.s.n_proc))
    lib().orc_rates_at_energy(C.byref(m.s), len(e), _p(e, PD), _p(out, PD))
    return out


def swarm(gas: dict, EN_Td: float, n0: int, n_steps: int, dt: float, seed: int,
          n_lo: int = 1000, n_hi: int = 1_000_000, kT_eV: float = 1.0, cap: int | None = None,
          E_override: float | None = None):
    """Runs a swarm; returns (moments [n_steps][16], counts [n_steps], coefficients [24])."""
    E = EN_Td * 1e-21 * gas["n_gas"] if E_override is None else E_override
    m = Model(gas, dt, seed, 64, None, None, E0=(0.0, 0.0, -E))
    if cap is None:
        cap = max(4 * n_hi, 4 * n0)
    p = Particles(cap)
    cfg = SwarmCfg(n0, n_lo, n_hi, n_steps, kT_eV)
    mom = np.zeros((n_steps, NMOM))
    counts = np.zeros(n_steps, np.int64)
    rc = lib().orc_swarm_run(C.byref(m.s), C.byref(cfg), C.byref(p.c), _p(mom, PD),
                             counts.ctypes.data_as(C.POINTER(C.c_longlong)))
    if rc:
        raise RuntimeError(f"orc_swarm_run failed rc={rc}")
    res = np.full(NRES, np.nan)
    i0 = n_steps // 4
    lib().orc_swarm_coefficients(_p(mom, PD), n_steps, i0, dt, gas["n_gas"], _p(res, PD))
    res[22] = p.n
    res[23] = mom[-1, 0]
    return mom, counts, res, m


RES_NAMES = ("W_flux", "W_bulk", "DL_flux", "DT_flux", "DL_bulk", "DT_bulk", "mean_eps",
             "k_ion", "k_att", "alpha", "eta")


def photon_draws(m: "Model", pid: int, step: int, n: int):
    """n photon draws of electron id pid at step `step` (draw indices 1..n):
    (emitted [n] bool, distance [n] m, direction [n][3])."""
    em = np.zeros(n, np.int32)
    r = np.zeros(n)
    d = np.zeros((n, 3))
    lib().orc_photon_draws(C.byref(m.s), C.c_uint64(pid), step, n, _p(em, PINT), _p(r, PD), _p(d, PD))
    return em.astype(bool), r, d
