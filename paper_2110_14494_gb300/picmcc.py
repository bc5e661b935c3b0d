"""Python binding of libpicmcc.so (include/picmcc.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory (workspaces, grids) and the
stream.  The functions keep the C names; thin classes below own the
workspace and the host arrays a context must keep alive.

The library must have been built (``paper_2110_14494_gb300.build.build()``);
importing this module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpicmcc.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CUDA, PIC_ERR_CAPACITY, PIC_ERR_OVERFLOW, PIC_ERR_TIMEOUT, PIC_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
PIC_MAX_PROC, PIC_SWARM_NMOM, PIC_SWARM_NRES = 16, 16, 24
RES_NAMES = ("W_flux", "W_bulk", "DL_flux", "DT_flux", "DL_bulk", "DT_bulk", "mean_eps", "k_ion", "k_att",
             "alpha", "eta")

PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
PU64 = C.POINTER(C.c_uint64)
VP = C.c_void_p


class pic_gas(C.Structure):
    _fields_ = [("n_proc", C.c_int), ("n_bins", C.c_int), ("eps", PD), ("sigma", PD), ("kind", PI),
                ("threshold", PD), ("density", PD), ("mass", PD), ("species", PI)]


class pic_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("origin", C.c_double * 3), ("capacity", C.c_longlong), ("seed", C.c_ulonglong),
                ("dt", C.c_double), ("gas", pic_gas), ("n_ppc", C.c_int), ("w_min", C.c_double),
                ("growth_trigger", C.c_double), ("particle_cap", C.c_longlong), ("boundary", C.c_int),
                ("sort_interval", C.c_int), ("coupled", C.c_int), ("v_lo", C.c_double), ("v_hi", C.c_double),
                ("v_mask", C.c_double), ("poisson_rtol", C.c_double), ("poisson_max_cycles", C.c_int),
                ("adaptive_dt", C.c_int), ("cfl", C.c_double), ("mobility", C.c_double),
                ("max_growth", C.c_double), ("photo_xi", C.c_double), ("photo_pq", C.c_double),
                ("pressure", C.c_double), ("p_o2", C.c_double), ("chi_min", C.c_double), ("chi_max", C.c_double),
                ("geometry", C.c_int), ("weight_interval", C.c_int)]


# Zheleznyak's absorption coefficients, 0.035 and 2 per (mm Torr), in 1/(m Pa)
TORR = 101325.0 / 760.0
ZHELEZNYAK_CHI_MIN = 0.035 / (1e-3 * TORR)
ZHELEZNYAK_CHI_MAX = 2.0 / (1e-3 * TORR)
K_BOLTZMANN = 1.380649e-23


def gas_pressure(n_gas: float, T: float = 300.0) -> float:
    """Ideal-gas pressure (Pa) of number density n_gas (m^-3) at temperature T (K)."""
    return n_gas * K_BOLTZMANN * T


class pic_particles_host(C.Structure):
    _fields_ = [(k, PD) for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "w")] + [("id", PU64)]


class pic_step_stats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in ("n_start", "n_end", "n_events", "n_null")] + \
               [("n_coll", C.c_longlong * PIC_MAX_PROC)] + \
               [(k, C.c_longlong) for k in ("n_children", "n_attached", "n_absorbed", "n_clamped",
                                            "n_processed", "n_weight_updates", "n_sorts")] + \
               [("w_ion", C.c_double), ("w_att", C.c_double), ("w_absorbed", C.c_double),
                ("poisson_cycles", C.c_int), ("poisson_rel_res", C.c_double), ("dt_last", C.c_double),
                ("t_total", C.c_double), ("ne_max", C.c_double), ("n_photo", C.c_longlong)]


class pic_profile_times(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("ms_push", "ms_children", "ms_field", "ms_reorder")] + \
               [(k, C.c_longlong) for k in ("n_push", "n_children", "n_field", "n_reorder", "n_launches",
                                            "n_speculative", "n_undone", "n_overlapped")]


class poisson_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("v_lo", C.c_double),
                ("v_hi", C.c_double), ("v_mask", C.c_double), ("precision", C.c_int)]


class poisson_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("rel_res", C.c_double)]


class swarm_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("gas", pic_gas), ("n_gas", C.c_double), ("n0", C.c_longlong),
                ("n_lo", C.c_longlong), ("n_hi", C.c_longlong), ("capacity", C.c_longlong),
                ("n_steps", C.c_int), ("dt", C.c_double), ("kT_eV", C.c_double), ("seed", C.c_ulonglong),
                ("sample_from", C.c_double), ("batched", C.c_int), ("block", C.c_int),
                ("blocks_per_sm", C.c_int), ("use_graph", C.c_int), ("warp_chunk", C.c_int)]


class swarm_result(C.Structure):
    _fields_ = [("v", C.c_double * PIC_SWARM_NRES)]


EXPORTS = ("pic_workspace_bytes", "pic_init", "pic_destroy", "pic_last_error", "pic_status_string",
           "pic_seed_gaussian", "pic_set_particles", "pic_get_particles", "pic_set_field", "pic_set_field_f64", "pic_step",
           "pic_deposit", "pic_weight_update", "pic_count", "pic_save", "pic_load", "pic_progress",
           "pic_profile", "pic_upload", "pic_download", "pic_set_poisson", "pic_get_field", "pic_get_deposit", "pic_set_multigrid",
           "poisson_workspace_bytes", "poisson_solve", "poisson_solve_noalloc", "swarm_workspace_bytes",
           "swarm_run", "swarm_autotune", "mlp_workspace_bytes", "mlp_forward", "mlp_forward_variant", "mlp_loss_grad",
           "mlp_fold_standardization", "mlp_features",
           "mlp_train", "poisson_axi_workspace_bytes", "poisson_axi_solve")

_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2110_14494_gb300.build.build() "
                           "(nvcc, sm_103a); there is no fallback")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    L.pic_workspace_bytes.argtypes = [P(pic_config)]
    L.pic_workspace_bytes.restype = C.c_size_t
    L.pic_init.argtypes = [P(pic_config), VP, C.c_size_t, VP, VP, P(VP)]
    L.pic_destroy.argtypes = [VP]
    L.pic_destroy.restype = None
    L.pic_last_error.argtypes = [VP]
    L.pic_last_error.restype = C.c_char_p
    L.pic_status_string.argtypes = [C.c_int]
    L.pic_status_string.restype = C.c_char_p
    L.pic_seed_gaussian.argtypes = [VP, C.c_double, C.c_double, PD, C.c_double, P(C.c_longlong)]
    L.pic_set_particles.argtypes = [VP, C.c_longlong, P(pic_particles_host), C.c_int]
    L.pic_get_particles.argtypes = [VP, P(pic_particles_host), C.c_longlong, P(C.c_longlong)]
    L.pic_set_field.argtypes = [VP, VP, VP, VP, PD]
    L.pic_set_field_f64.argtypes = [VP, VP, VP, VP, PD]
    L.pic_step.argtypes = [VP, C.c_int, P(pic_step_stats)]
    L.pic_set_poisson.argtypes = [VP, C.c_double, C.c_int, C.c_int]
    L.pic_set_multigrid.argtypes = [VP, C.c_int, C.c_int]
    L.pic_deposit.argtypes = [VP, VP, VP, VP, VP]
    L.pic_get_deposit.argtypes = [VP, VP, VP, VP]
    L.pic_get_field.argtypes = [VP, VP, VP, VP]
    L.pic_weight_update.argtypes = [VP]
    L.pic_count.argtypes = [VP, P(C.c_longlong)]
    L.pic_save.argtypes = [VP, VP, P(C.c_size_t)]
    L.pic_load.argtypes = [VP, VP, C.c_size_t]
    L.pic_progress.argtypes = [VP, P(C.c_longlong), P(C.c_longlong), P(C.c_longlong)]
    L.pic_profile.argtypes = [VP, C.c_int, P(pic_profile_times)]
    L.pic_upload.argtypes = [VP, C.c_longlong, P(VP), C.c_int]
    L.pic_download.argtypes = [VP, P(VP), C.c_longlong, P(C.c_longlong)]
    L.poisson_workspace_bytes.argtypes = [P(poisson_config)]
    L.poisson_workspace_bytes.restype = C.c_size_t
    L.poisson_solve.argtypes = [P(poisson_config), VP, VP, VP, VP, VP, VP, C.c_double, C.c_int, VP, C.c_size_t,
                                P(poisson_stats), VP]
    L.poisson_solve_noalloc.argtypes = [P(poisson_config), VP, VP, VP, VP, VP, VP, C.c_double, C.c_int,
                                        P(poisson_stats), VP]
    L.swarm_workspace_bytes.argtypes = [P(swarm_config), C.c_int]
    L.swarm_workspace_bytes.restype = C.c_size_t
    L.swarm_run.argtypes = [P(swarm_config), C.c_int, PD, PD, VP, C.c_size_t, P(swarm_result), PD,
                            P(C.c_longlong), VP]
    L.swarm_autotune.argtypes = [P(swarm_config), C.c_int, PD, PD, VP, C.c_size_t, P(C.c_int), P(C.c_int),
                                 P(C.c_int), P(C.c_int), PD, VP]
    L.poisson_axi_workspace_bytes.argtypes = [C.c_int, C.c_int]
    L.poisson_axi_workspace_bytes.restype = C.c_size_t
    L.poisson_axi_solve.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, VP, VP, VP, VP,
                                    VP, C.c_double, C.c_int, VP, C.c_size_t, P(poisson_stats), VP]
    L.mlp_workspace_bytes.argtypes = [C.c_int]
    L.mlp_workspace_bytes.restype = C.c_size_t
    L.mlp_forward.argtypes = [VP, VP, VP, C.c_longlong, VP, C.c_size_t, VP]
    L.mlp_fold_standardization.argtypes = [VP, PD, PD, PD, PD, VP, VP]
    L.mlp_features.argtypes = [VP, VP, VP, C.c_longlong, VP]
    L.mlp_forward_variant.argtypes = [VP, VP, VP, C.c_longlong, C.c_int, VP, C.c_size_t, VP]
    L.mlp_loss_grad.argtypes = [VP, VP, VP, C.c_int, VP, VP, VP, C.c_size_t, VP]
    L.mlp_train.argtypes = [VP, VP, VP, C.c_int, VP, VP, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                            C.c_float, VP, VP, C.c_size_t, VP]
    _lib = L
    return L


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _check(rc, ctx=None, what=""):
    if rc != PIC_OK:
        msg = lib().pic_last_error(ctx).decode() if ctx else lib().pic_status_string(rc).decode()
        raise PicError(rc, f"{what}: {msg}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class HostSet:
    """Host arrays of pic_upload / pic_download checked once (see
    _host_arrays): the pointers are kept with references to the arrays."""

    def __init__(self, arrays, capacity: int, precision: int):
        self.ptrs = _host_arrays(arrays, capacity, precision, "host set")
        self.capacity = int(capacity)
        self.precision = int(precision)
        self._keep = list(arrays)


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _host_arrays(arrays, count: int, precision: int, what: str):
    """Pointers of the 11 host arrays of pic_upload / pic_download (x, y, z,
    vx, vy, vz, ax, ay, az, w in the context precision, then 64-bit ids),
    after checking that each is a contiguous host array of that type holding
    at least `count` entries: the library reads or writes that many through
    the raw pointers."""
    if len(arrays) != 11:
        raise ValueError(f"{what}: 11 arrays expected, got {len(arrays)}")
    real = np.float32 if precision == 32 else np.float64
    ptrs = []
    for i, a in enumerate(arrays):
        ok_types = (real,) if i < 10 else (np.int64, np.uint64)
        if hasattr(a, "data_ptr"):  # a torch tensor
            import torch
            tmap = {np.float32: torch.float32, np.float64: torch.float64, np.int64: torch.int64,
                    np.uint64: getattr(torch, "uint64", torch.int64)}
            good = (a.device.type == "cpu" and a.is_contiguous() and a.dtype in [tmap[t] for t in ok_types]
                    and a.numel() >= count)
            ptr = a.data_ptr()
        else:
            good = (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype.type in ok_types
                    and a.size >= count)
            ptr = a.ctypes.data if isinstance(a, np.ndarray) else 0
        if not good:
            kind = "float%d" % precision if i < 10 else "int64/uint64"
            raise ValueError(f"{what}: array {i} must be a contiguous host {kind} array of at least {count} entries")
        ptrs.append(ptr)
    return (VP * 11)(*ptrs)


def _workspace(nbytes: int):
    import torch
    t = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device="cuda")
    off = (-t.data_ptr()) % 256
    return t, t.data_ptr() + off


class Gas:
    """Keeps the host arrays of a pic_gas alive."""

    def __init__(self, gas: dict):
        self.arrays = dict(
            eps=np.ascontiguousarray(gas["eps"], np.float64),
            sigma=np.ascontiguousarray(gas["sigma"], np.float64),
            kind=np.ascontiguousarray(gas["kind"], np.int32),
            threshold=np.ascontiguousarray(gas["threshold"], np.float64),
            density=np.ascontiguousarray(gas["density"], np.float64),
            mass=np.ascontiguousarray(gas["mass"], np.float64))
        if gas.get("species") is not None:
            self.arrays["species"] = np.ascontiguousarray(gas["species"], np.int32)
        a = self.arrays
        self.c = pic_gas(a["sigma"].shape[0], a["sigma"].shape[1], a["eps"].ctypes.data_as(PD),
                         a["sigma"].ctypes.data_as(PD), a["kind"].ctypes.data_as(PI),
                         a["threshold"].ctypes.data_as(PD), a["density"].ctypes.data_as(PD),
                         a["mass"].ctypes.data_as(PD),
                         a["species"].ctypes.data_as(PI) if "species" in a else None)
        self.n_gas = float(gas.get("n_gas", 0.0))


class PicContext:
    """A pic_ctx over a torch-allocated workspace."""

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "w")

    def __init__(self, gas: dict, grid: dict, *, precision=32, capacity=1 << 20, seed=1, dt=1e-12, mask=None,
                 n_ppc=75, w_min=1.0, growth_trigger=0.0, particle_cap=0, boundary=0, sort_interval=0,
                 coupled=False, v_lo=0.0, v_hi=0.0, v_mask=0.0, poisson_rtol=1e-6, poisson_max_cycles=100,
                 adaptive_dt=False, cfl=0.5, mobility=0.06, max_growth=1.2, photo_xi=0.0, photo_pq=4000.0,
                 pressure=None, p_o2=None, chi_min=ZHELEZNYAK_CHI_MIN, chi_max=ZHELEZNYAK_CHI_MAX, geometry=0,
                 weight_interval=0, stream=None):
        import torch
        self.gas = Gas(gas)
        c = pic_config()
        c.precision, c.nx, c.ny, c.nz, c.dx = precision, grid["nx"], grid["ny"], grid["nz"], grid["dx"]
        for d in range(3):
            c.origin[d] = grid["origin"][d]
        c.capacity, c.seed, c.dt, c.gas = capacity, seed, dt, self.gas.c
        c.n_ppc, c.w_min, c.growth_trigger, c.particle_cap = n_ppc, w_min, growth_trigger, particle_cap
        c.boundary, c.sort_interval, c.coupled = boundary, sort_interval, int(coupled)
        c.v_lo, c.v_hi, c.v_mask, c.poisson_rtol, c.poisson_max_cycles = v_lo, v_hi, v_mask, poisson_rtol, \
            poisson_max_cycles
        c.adaptive_dt, c.cfl, c.mobility, c.max_growth = int(adaptive_dt), cfl, mobility, max_growth
        # photoionization: pressure from the gas density at 300 K unless given; p_O2 = 20 % of it
        p = pressure if pressure is not None else gas_pressure(float(gas["n_gas"]))
        c.photo_xi, c.photo_pq, c.pressure = photo_xi, photo_pq, p
        c.p_o2 = p_o2 if p_o2 is not None else 0.2 * p
        c.chi_min, c.chi_max = chi_min, chi_max
        c.geometry, c.weight_interval = geometry, weight_interval
        self.cfg = c
        self.grid = grid
        self.ncell = grid["nx"] * grid["ny"] * grid["nz"]
        nbytes = lib().pic_workspace_bytes(C.byref(c))
        if nbytes == 0:
            raise PicError(PIC_ERR_ARG, "invalid pic_config")
        self.ws_bytes = nbytes
        self._ws, self._ws_ptr = _workspace(nbytes)
        self.mask = None
        if mask is not None:
            self.mask = torch.as_tensor(np.ascontiguousarray(mask, np.uint8)).cuda()
        self.stream = stream
        h = C.c_void_p()
        _check(lib().pic_init(C.byref(c), C.c_void_p(self._ws_ptr), nbytes, _ptr(self.mask), _stream(stream),
                              C.byref(h)), None, "pic_init")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seed_gaussian(self, n0, radius, center, w0) -> int:
        cen = (C.c_double * 3)(*center)
        n = C.c_longlong()
        _check(lib().pic_seed_gaussian(self.h, n0, radius, cen, w0, C.byref(n)), self.h, "pic_seed_gaussian")
        return n.value

    def set_particles(self, p: dict, accel_valid=False):
        n = len(p["x"])
        keep = {k: np.ascontiguousarray(p[k], np.float64) for k in self.FIELDS if k in p}
        ids = np.ascontiguousarray(p["id"], np.uint64)
        if any(a.shape != (n,) for a in keep.values()) or ids.shape != (n,):
            raise ValueError("set_particles: every field must be a 1-D array of len(p['x']) entries")
        hp = pic_particles_host(*[keep[k].ctypes.data_as(PD) if k in keep else None for k in self.FIELDS],
                                ids.ctypes.data_as(PU64))
        _check(lib().pic_set_particles(self.h, n, C.byref(hp), int(accel_valid)), self.h, "pic_set_particles")

    def get_particles(self) -> dict:
        n = C.c_longlong()
        _check(lib().pic_get_particles(self.h, None, 0, C.byref(n)), self.h, "pic_get_particles")
        out = {k: np.zeros(n.value) for k in self.FIELDS}
        out["id"] = np.zeros(n.value, np.uint64)
        hp = pic_particles_host(*[out[k].ctypes.data_as(PD) for k in self.FIELDS], out["id"].ctypes.data_as(PU64))
        _check(lib().pic_get_particles(self.h, C.byref(hp), n.value, C.byref(n)), self.h, "pic_get_particles")
        return out

    def set_field(self, Ex=None, Ey=None, Ez=None, uniform=None):
        """Cell-centred field grids [nz][ny][nx] as contiguous CUDA tensors, all float32
        (pic_set_field) or all float64 (pic_set_field_f64); or a uniform field."""
        u = (C.c_double * 3)(*(uniform if uniform is not None else (0.0, 0.0, 0.0)))
        if Ex is None:
            _check(lib().pic_set_field(self.h, None, None, None, u), self.h, "pic_set_field")
            return
        import torch
        n = self.grid["nx"] * self.grid["ny"] * self.grid["nz"]
        for f in (Ex, Ey, Ez):
            if (not isinstance(f, torch.Tensor) or not f.is_cuda or not f.is_contiguous() or f.numel() != n or
                    f.dtype != Ex.dtype or f.dtype not in (torch.float32, torch.float64)):
                raise TypeError("field grids: three contiguous CUDA tensors of %d float32 or float64 values" % n)
        fn = "pic_set_field" if Ex.dtype == torch.float32 else "pic_set_field_f64"
        _check(getattr(lib(), fn)(self.h, _ptr(Ex), _ptr(Ey), _ptr(Ez), u), self.h, fn)

    def step(self, n_steps=1, stats=False):
        st = pic_step_stats() if stats else None
        _check(lib().pic_step(self.h, n_steps, C.byref(st) if st is not None else None), self.h, "pic_step")
        return st

    def deposit(self, q_e=None, q_pos=None, q_neg=None, rho=None):
        _check(lib().pic_deposit(self.h, _ptr(q_e), _ptr(q_pos), _ptr(q_neg), _ptr(rho)), self.h, "pic_deposit")

    def get_deposit(self, q_e=None, q_pos=None, q_neg=None):
        """The fixed-point grids as the last step left them (int64 CUDA tensors), no new deposit."""
        _check(lib().pic_get_deposit(self.h, _ptr(q_e), _ptr(q_pos), _ptr(q_neg)), self.h, "pic_get_deposit")

    def get_field(self, Ex=None, Ey=None, Ez=None):
        """The field the next gather reads, into float64 CUDA tensors [nz][ny][nx] (new ones if none given)."""
        import torch
        if Ex is None and Ey is None and Ez is None:
            shape = (self.grid["nz"], self.grid["ny"], self.grid["nx"])
            Ex, Ey, Ez = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3))
        _check(lib().pic_get_field(self.h, _ptr(Ex), _ptr(Ey), _ptr(Ez)), self.h, "pic_get_field")
        return Ex, Ey, Ez

    def weight_update(self):
        _check(lib().pic_weight_update(self.h), self.h, "pic_weight_update")

    def count(self) -> int:
        n = C.c_longlong()
        _check(lib().pic_count(self.h, C.byref(n)), self.h, "pic_count")
        return n.value

    def progress(self):
        u, p, s = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib().pic_progress(self.h, C.byref(u), C.byref(p), C.byref(s)), self.h, "pic_progress")
        return u.value, p.value, s.value

    def set_poisson(self, rtol, max_cycles, device_loop=True):
        """Coupled solve settings: residual target, V-cycle limit, and whether
        float32 contexts run the CG loop on the device (graph conditional
        nodes) or check the residual from the host after every iteration."""
        _check(lib().pic_set_poisson(self.h, float(rtol), int(max_cycles), int(bool(device_loop))), self.h,
               "pic_set_poisson")

    def set_multigrid(self, pre_sweeps=2, post_sweeps=2):
        """Smoothing sweeps of the coupled solve's V-cycle preconditioner (Cartesian contexts)."""
        _check(lib().pic_set_multigrid(self.h, int(pre_sweeps), int(post_sweeps)), self.h, "pic_set_multigrid")

    def profile(self, enable=True):
        t = pic_profile_times()
        _check(lib().pic_profile(self.h, int(enable), C.byref(t)), self.h, "pic_profile")
        return {f[0]: getattr(t, f[0]) for f in pic_profile_times._fields_}

    def host_set(self, arrays, capacity):
        """The 11 host arrays validated once (type, contiguity, at least
        `capacity` entries) for repeated upload / download calls."""
        return HostSet(arrays, capacity, self.cfg.precision)

    def upload(self, arrays, n, accel_valid=True):
        """arrays: 11 host tensors/arrays (pinned for asynchronous copies) in native precision, or a HostSet."""
        if isinstance(arrays, HostSet):
            if arrays.precision != self.cfg.precision or not 0 <= n <= arrays.capacity:
                raise ValueError("pic_upload: host set of another precision or smaller than n")
            ptrs = arrays.ptrs
        else:
            ptrs = _host_arrays(arrays, n, self.cfg.precision, "pic_upload")
        _check(lib().pic_upload(self.h, n, ptrs, int(accel_valid)), self.h, "pic_upload")

    def download(self, arrays, cap=None) -> int:
        if isinstance(arrays, HostSet):
            if arrays.precision != self.cfg.precision:
                raise ValueError("pic_download: host set of another precision")
            ptrs, cap = arrays.ptrs, arrays.capacity if cap is None else min(cap, arrays.capacity)
        else:
            ptrs = _host_arrays(arrays, cap, self.cfg.precision, "pic_download")
        n = C.c_longlong()
        _check(lib().pic_download(self.h, ptrs, cap, C.byref(n)), self.h, "pic_download")
        return n.value

    def save(self) -> bytes:
        sz = C.c_size_t(0)
        _check(lib().pic_save(self.h, None, C.byref(sz)), self.h, "pic_save")
        buf = (C.c_char * sz.value)()
        _check(lib().pic_save(self.h, buf, C.byref(sz)), self.h, "pic_save")
        return bytes(buf)

    def load(self, blob: bytes):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        _check(lib().pic_load(self.h, buf, len(blob)), self.h, "pic_load")


def poisson_solve(grid: dict, rho, phi, mask=None, E=None, v_lo=0.0, v_hi=0.0, v_mask=0.0, rtol=1e-6,
                  max_cycles=100, stream=None, precision=64):
    """rho, phi: float64 CUDA tensors [nz][ny][nx]; E: optional tuple of three float32 tensors.
    precision 64: CG in float64; 32: float-pair potential with float32 CG and refinement."""
    pc = poisson_config(grid["nx"], grid["ny"], grid["nz"], grid["dx"], v_lo, v_hi, v_mask, precision)
    nb = lib().poisson_workspace_bytes(C.byref(pc))
    ws, ptr = _workspace(nb)
    st = poisson_stats()
    Ex, Ey, Ez = E if E is not None else (None, None, None)
    rc = lib().poisson_solve(C.byref(pc), _ptr(rho), _ptr(mask), _ptr(phi), _ptr(Ex), _ptr(Ey), _ptr(Ez), rtol,
                             max_cycles, C.c_void_p(ptr), nb, C.byref(st), _stream(stream))
    _check(rc, None, "poisson_solve")
    return st.cycles, st.rel_res


def poisson_axi_solve(nr: int, nz: int, dx: float, rho, phi, mask=None, E=None, v_lo=0.0, v_hi=0.0, v_mask=0.0,
                      rtol=1e-6, max_cycles=100, stream=None):
    """Axisymmetric solve; rho, phi: float64 CUDA tensors [nz][nr]; E: optional (Er, Ez) float32 tensors."""
    nb = lib().poisson_axi_workspace_bytes(nr, nz)
    if nb == 0:
        raise PicError(PIC_ERR_ARG, "poisson_axi_solve: unsupported grid")
    ws, ptr = _workspace(nb)
    st = poisson_stats()
    Er, Ez = E if E is not None else (None, None)
    rc = lib().poisson_axi_solve(nr, nz, dx, v_lo, v_hi, v_mask, _ptr(rho), _ptr(mask), _ptr(phi), _ptr(Er),
                                 _ptr(Ez), rtol, max_cycles, C.c_void_p(ptr), nb, C.byref(st), _stream(stream))
    _check(rc, None, "poisson_axi_solve")
    return st.cycles, st.rel_res


def _swarm_cfg(gas, precision, n0, n_steps, dt, kT_eV, seed, n_lo, n_hi, capacity, sample_from, batched, block,
               blocks_per_sm, use_graph, warp_chunk=0):
    g = Gas(gas)
    if capacity is None:
        capacity = max(2 * n_hi, 4 * n0)
    sc = swarm_config(precision, g.c, g.n_gas, n0, n_lo, n_hi, capacity, n_steps, dt, kT_eV, seed, sample_from,
                      int(batched), block, blocks_per_sm, int(use_graph), int(warp_chunk))
    return g, sc


def _o2(o2_frac, n):
    if o2_frac is None:
        return None
    f = np.ascontiguousarray(np.broadcast_to(np.asarray(o2_frac, np.float64), (n,)))
    return f


def swarm_autotune(gas: dict, EN_Td, *, o2_frac=None, precision=32, n0=10000, n_steps=100, dt=1e-12, kT_eV=1.0,
                   seed=1, n_lo=1000, n_hi=1_000_000, capacity=None, stream=None):
    """Returns (block, blocks_per_sm, warp_chunk, use_graph, ms_per_step) of the fastest batched launch shape."""
    EN = np.ascontiguousarray(np.atleast_1d(EN_Td), np.float64)
    f = _o2(o2_frac, len(EN))
    g, sc = _swarm_cfg(gas, precision, n0, n_steps, dt, kT_eV, seed, n_lo, n_hi, capacity, 0.25, True, 0, 0, 1)
    nb = lib().swarm_workspace_bytes(C.byref(sc), len(EN))
    if nb == 0:
        raise PicError(PIC_ERR_ARG, "invalid swarm_config")
    ws, ptr = _workspace(nb)
    b, bps, ch, mode, ms = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
    _check(lib().swarm_autotune(C.byref(sc), len(EN), EN.ctypes.data_as(PD), f.ctypes.data_as(PD) if f is not None
                                else None, C.c_void_p(ptr), nb, C.byref(b), C.byref(bps), C.byref(ch), C.byref(mode),
                                C.byref(ms), _stream(stream)), None, "swarm_autotune")
    return b.value, bps.value, ch.value, mode.value, ms.value


def swarm_run(gas: dict, EN_Td, *, o2_frac=None, precision=64, n0=10000, n_steps=2000, dt=1e-12, kT_eV=1.0, seed=1,
              n_lo=1000, n_hi=1_000_000, capacity=None, sample_from=0.25, stream=None, want_moments=False,
              batched=False, block=0, blocks_per_sm=0, use_graph=2, warp_chunk=0):
    """Runs len(EN_Td) swarms; returns (results [n][24], moments or None, counts or None).
    o2_frac: per-swarm O2 fractions (a scalar applies to all; needs the gas's species); use_graph (batched):
    0 kernels per step, 1 step graph replayed, 2 one persistent launch (block = 0: autotuned with the shape)."""
    EN = np.ascontiguousarray(np.atleast_1d(EN_Td), np.float64)
    f = _o2(o2_frac, len(EN))
    g, sc = _swarm_cfg(gas, precision, n0, n_steps, dt, kT_eV, seed, n_lo, n_hi, capacity, sample_from, batched,
                       block, blocks_per_sm, use_graph, warp_chunk)
    nb = lib().swarm_workspace_bytes(C.byref(sc), len(EN))
    if nb == 0:
        raise PicError(PIC_ERR_ARG, "invalid swarm_config")
    ws, ptr = _workspace(nb)
    res = (swarm_result * len(EN))()
    mom = np.zeros((len(EN), n_steps, PIC_SWARM_NMOM)) if want_moments else None
    cnt = np.zeros((len(EN), n_steps), np.int64) if want_moments else None
    rc = lib().swarm_run(C.byref(sc), len(EN), EN.ctypes.data_as(PD), f.ctypes.data_as(PD) if f is not None else None,
                         C.c_void_p(ptr), nb, res, mom.ctypes.data_as(PD) if mom is not None else None,
                         cnt.ctypes.data_as(C.POINTER(C.c_longlong)) if cnt is not None else None, _stream(stream))
    _check(rc, None, "swarm_run")
    out = np.array([[r.v[i] for i in range(PIC_SWARM_NRES)] for r in res])
    return out, mom, cnt


MLP_NI, MLP_NH, MLP_NO, MLP_NPARAMS = 2, 128, 6, 17670


def _mlp_ws(n):
    nb = lib().mlp_workspace_bytes(n)
    if nb == 0:
        raise PicError(PIC_ERR_ARG, f"mlp: unsupported batch size {n}")
    return _workspace(nb)


def mlp_forward(params, x, y=None, stream=None, variant=0):
    """params: float32 CUDA [17670]; x: float32 CUDA [n][2] (standardized); returns y [n][6].
    variant 0: tcgen05 kernel; 1: mma.sync kernel."""
    import torch
    n = int(x.shape[0])
    if y is None:
        y = torch.empty((n, MLP_NO), dtype=torch.float32, device=x.device)
    ws, ptr = _mlp_ws(0)
    _check(lib().mlp_forward_variant(_ptr(params), _ptr(x), _ptr(y), n, int(variant), C.c_void_p(ptr),
                                     lib().mlp_workspace_bytes(0), _stream(stream)), None, "mlp_forward")
    return y


def mlp_fold_standardization(params, x_mean, x_scale, y_mean, y_scale, out=None, stream=None):
    """Parameters of the network on raw inputs and targets (mlp_fold_standardization)."""
    import torch
    if out is None:
        out = torch.empty_like(params)
    arr = lambda v, m: (C.c_double * m)(*[float(a) for a in np.asarray(v, np.float64).ravel()[:m]])
    _check(lib().mlp_fold_standardization(_ptr(params), arr(x_mean, MLP_NI), arr(x_scale, MLP_NI),
                                          arr(y_mean, MLP_NO), arr(y_scale, MLP_NO), _ptr(out), _stream(stream)),
           None, "mlp_fold_standardization")
    return out


def mlp_features(EN_Td, f_o2, x=None, stream=None):
    """Network inputs (log10 E/N, O2 fraction) as float32 [n][2] from float64 CUDA tensors."""
    import torch
    n = int(EN_Td.shape[0])
    if x is None:
        x = torch.empty((n, MLP_NI), dtype=torch.float32, device=EN_Td.device)
    _check(lib().mlp_features(_ptr(EN_Td), _ptr(f_o2), _ptr(x), n, _stream(stream)), None, "mlp_features")
    return x


def mlp_loss_grad(params, x, t, stream=None):
    """Returns (loss tensor [1], grad tensor [17670]) on the device."""
    import torch
    n = int(x.shape[0])
    g = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    ws, ptr = _mlp_ws(n)
    _check(lib().mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), n, _ptr(g), _ptr(loss), C.c_void_p(ptr),
                               lib().mlp_workspace_bytes(n), _stream(stream)), None, "mlp_loss_grad")
    return loss, g


def mlp_train(params, m, v, step0, x, t, n_steps, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """n_steps full-batch Adam steps in place on params, m, v; returns the loss tensor [1]."""
    import torch
    n = int(x.shape[0])
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    ws, ptr = _mlp_ws(n)
    _check(lib().mlp_train(_ptr(params), _ptr(m), _ptr(v), int(step0), _ptr(x), _ptr(t), n, int(n_steps), lr,
                           beta1, beta2, eps, _ptr(loss), C.c_void_p(ptr), lib().mlp_workspace_bytes(n),
                           _stream(stream)), None, "mlp_train")
    return loss
