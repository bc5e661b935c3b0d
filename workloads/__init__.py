"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates inputs*: cross-section tables, particle states,
electric fields, charge densities and the electrode mask. It holds none of
the method's arithmetic (no rate tables, no pushes, no deposits, no solves);
each side (the CPU oracle and the CUDA library) does that on its own.

The gas and the workloads follow the paper's conditions: artificial air with
80 % N2 and 20 % O2 (Sec. 2.3), cross sections tabulated on log-spaced energy
bins (Sec. 2.1.5 describes tabulated cross-section input; the magnitudes here
are synthetic analytic stand-ins because the Phelps data is not available),
a rod electrode with a hemispherical cap (Sec. 2.3) and a Gaussian neutral
seed at the electrode tip (Eq. 7).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2110144940

# Process kinds, shared as plain integers with both implementations.
ELASTIC, EXCITATION, IONIZATION, ATTACHMENT = 0, 1, 2, 3
# Target species of a process (for per-swarm O2 fractions).
N2, O2 = 0, 1

AMU_KG = 1.66053906660e-27          # CODATA 2018 atomic mass unit
M_N2_KG = 28.0134 * AMU_KG
M_O2_KG = 31.9988 * AMU_KG

# Gas number density used by the workloads (stated for 300 K and 1 bar).
N_GAS = 2.45e25
# Density the paper uses for its kV/cm <-> Td conversion (Sec. 2.3).
N_GAS_PAPER = 2.414e25


def log_nodes(n_bins: int = 1000, eps_min: float = 0.01, eps_max: float = 1000.0) -> np.ndarray:
    """Energies (eV) of the table nodes, uniform in ln(eps) from eps_min to eps_max."""
    j = np.arange(n_bins, dtype=np.float64)
    return eps_min * np.power(eps_max / eps_min, j / (n_bins - 1))


def _lnx_over_x(eps: np.ndarray, thr: float) -> np.ndarray:
    out = np.zeros_like(eps)
    m = eps > thr
    x = eps[m] / thr
    out[m] = np.log(x) / x
    return out


def synthetic_air(n_bins: int = 1000, eps_min: float = 0.01, eps_max: float = 1000.0,
                  n_gas: float = N_GAS, o2_frac: float = 0.2) -> dict:
    """Seven-process synthetic N2/O2 gas on log-spaced bins.

    Processes (analytic cross sections in m^2, x = eps/eps_th):
      0 elastic N2            1.0e-19 (1 + eps/10)^-1/2
      1 elastic O2            same form
      2 excitation N2 6.2 eV  2e-21  ln(x)/x
      3 excitation N2 11 eV   1.5e-20 ln(x)/x
      4 ionization N2 15.6 eV 6e-20  ln(x)/x
      5 ionization O2 12.06eV 7e-20  ln(x)/x
      6 attachment O2         1.3e-22 exp(-(eps-6.5)^2 / (2 0.7^2))
    Inelastic cross sections vanish below their threshold.
    """
    eps = log_nodes(n_bins, eps_min, eps_max)
    n_n2 = (1.0 - o2_frac) * n_gas
    n_o2 = o2_frac * n_gas
    el = 1.0e-19 / np.sqrt(1.0 + eps / 10.0)
    sig = np.stack([
        el,
        el.copy(),
        2e-21 * _lnx_over_x(eps, 6.2),
        1.5e-20 * _lnx_over_x(eps, 11.0),
        6e-20 * _lnx_over_x(eps, 15.6),
        7e-20 * _lnx_over_x(eps, 12.06),
        1.3e-22 * np.exp(-(eps - 6.5) ** 2 / (2 * 0.7 ** 2)),
    ])
    return dict(
        eps=eps,
        sigma=np.ascontiguousarray(sig),
        kind=np.array([ELASTIC, ELASTIC, EXCITATION, EXCITATION, IONIZATION, IONIZATION, ATTACHMENT],
                      dtype=np.int32),
        threshold=np.array([0.0, 0.0, 6.2, 11.0, 15.6, 12.06, 0.0]),
        density=np.array([n_n2, n_o2, n_n2, n_n2, n_n2, n_o2, n_o2]),
        mass=np.array([M_N2_KG, M_O2_KG, M_N2_KG, M_N2_KG, M_N2_KG, M_O2_KG, M_O2_KG]),
        species=np.array([N2, O2, N2, N2, N2, O2, O2], dtype=np.int32),
        n_gas=n_gas,
    )


def single_process_gas(kind: int, sigma_v: float, n_gas: float = N_GAS, mass: float = 0.0,
                       threshold: float = 0.0, n_bins: int = 64, eps_min: float = 0.01,
                       eps_max: float = 1000.0) -> dict:
    """A one-process gas whose tabulated N*sigma*v is (close to) a constant.

    `sigma_v` is the rate coefficient sigma*v in m^3/s; the cross section at
    node energy eps is sigma_v / v(eps) with v(eps) = sqrt(2 e eps / m_e).
    mass = 0 means an infinitely heavy target (no elastic energy loss).
    """
    e, me = 1.602176634e-19, 9.1093837015e-31
    eps = log_nodes(n_bins, eps_min, eps_max)
    v = np.sqrt(2.0 * e * eps / me)
    return dict(
        eps=eps,
        sigma=np.ascontiguousarray((sigma_v / v)[None, :]),
        kind=np.array([kind], dtype=np.int32),
        threshold=np.array([threshold]),
        density=np.array([n_gas]),
        mass=np.array([mass]),
        species=np.array([N2], dtype=np.int32),
        n_gas=n_gas,
    )


def multi_gas(parts: list[dict]) -> dict:
    """Concatenate the processes of several gases that share the same nodes."""
    eps = parts[0]["eps"]
    for p in parts:
        assert np.array_equal(p["eps"], eps)
    return dict(
        eps=eps,
        sigma=np.ascontiguousarray(np.concatenate([p["sigma"] for p in parts])),
        kind=np.concatenate([p["kind"] for p in parts]).astype(np.int32),
        threshold=np.concatenate([p["threshold"] for p in parts]),
        density=np.concatenate([p["density"] for p in parts]),
        mass=np.concatenate([p["mass"] for p in parts]),
        species=np.concatenate([p["species"] for p in parts]).astype(np.int32),
        n_gas=parts[0]["n_gas"],
    )


def zero_gas(n_bins: int = 16) -> dict:
    """A gas with one process of zero cross section: particles fly ballistically."""
    g = single_process_gas(ELASTIC, 0.0, n_bins=n_bins)
    g["sigma"][:] = 0.0
    return g


# --------------------------------------------------------------------------- grids

def grid_spec(nx: int, ny: int, nz: int, dx: float, origin=(0.0, 0.0, 0.0)) -> dict:
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), dx=float(dx), origin=tuple(float(o) for o in origin))


def needle_mask(g: dict, length: float, radius: float) -> np.ndarray:
    """uint8 [nz][ny][nx] mask of cells whose centre lies inside a rod electrode.

    The rod hangs from the top plate (z = L) at the centre of x and y, has the
    given radius, and ends in a hemispherical cap whose lowest point is at
    z = L - length (Sec. 2.3 describes a rod with a semi-spherical cap).
    """
    nx, ny, nz, dx = g["nx"], g["ny"], g["nz"], g["dx"]
    ox, oy, oz = g["origin"]
    xc = ox + (np.arange(nx) + 0.5) * dx
    yc = oy + (np.arange(ny) + 0.5) * dx
    zc = oz + (np.arange(nz) + 0.5) * dx
    cx, cy = ox + 0.5 * nx * dx, oy + 0.5 * ny * dx
    ztop = oz + nz * dx
    zcap = ztop - length + radius          # centre of the hemispherical cap
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    r2 = (X - cx) ** 2 + (Y - cy) ** 2
    rod = (r2 <= radius ** 2) & (Z >= zcap)
    cap = (r2 + (Z - zcap) ** 2) <= radius ** 2
    return np.ascontiguousarray((rod | cap).astype(np.uint8))


def streamer_full() -> dict:
    """The full-size streamer: a 10 mm plate-plate gap at 15.6 kV on 256 x 256 x
    512 cells of 19.53 um (5 x 5 x 10 mm), a 2 mm needle of 0.2 mm radius
    hanging from the top plate, photoionization on (xi = 0.075, p_q = 40 mbar,
    1 bar-equivalent density at 300 K, 20 % O2), up to 2e8 super-particles,
    dt <= 2 ps.  The seed is not specified for this case; it is the 128^3
    workload's Gaussian (peak 1e19 m^-3, 0.1 mm radius) at the needle tip."""
    dx = 10e-3 / 512
    g = grid_spec(256, 256, 512, dx)
    L = 512 * dx
    needle_len, needle_r = 2e-3, 0.2e-3
    tip = (0.5 * 256 * dx, 0.5 * 256 * dx, L - needle_len)
    return dict(grid=g, L=L, v_bottom=0.0, v_top=15.6e3, needle_length=needle_len, needle_radius=needle_r,
                seed_n0=1e19, seed_radius=1e-4, seed_center=tip, n_initial=1_000_000,
                particle_cap=200_000_000, dt=2e-12, n_ppc=75, w_min=1.0, growth_trigger=1.25,
                photo_xi=0.075, photo_pq=4000.0, t_end=15e-9)


def streamer_axi() -> dict:
    """Axisymmetric streamer in the paper's cylindrical domain (Sec. 2.3): 10 mm
    radius x 10 mm gap on 512 x 512 (r, z) cells of 19.53 um, a 2 mm rod of
    0.2 mm radius on the axis hanging from the top plate (tip near z = 7.8 mm),
    15.6 kV, the paper's seed (Eq. 7 read with a negative exponent: peak
    1e16 m^-3, 0.1 mm radius at the tip, weight-one particles), photoionization
    on, weight updates every 10 steps, dt <= 2 ps."""
    dx = 10e-3 / 512
    g = axi_grid(512, 512, dx)
    L = 512 * dx
    needle_len, needle_r = 2e-3, 0.2e-3
    return dict(grid=g, L=L, v_bottom=0.0, v_top=15.6e3, needle_length=needle_len, needle_radius=needle_r,
                seed_n0=1e16, seed_radius=1e-4, seed_center=(0.0, 0.0, L - needle_len), w0=1.0,
                particle_cap=20_000_000, dt=2e-12, n_ppc=75, w_min=1.0, growth_trigger=1.25, weight_interval=10,
                photo_xi=0.075, photo_pq=4000.0)


def streamer_128() -> dict:
    """The 128^3 streamer workload: 20 um cells, plates at 0 V / 5.12 kV (20 kV/cm),
    a 0.5 mm needle of 0.1 mm radius hanging from the top plate, a Gaussian
    seed of peak 1e19 m^-3 and 0.1 mm radius at the needle tip, 1e6 initial
    super-particles capped at 2e7, dt = 2 ps."""
    g = grid_spec(128, 128, 128, 20e-6)
    L = 128 * 20e-6
    needle_len, needle_r = 0.5e-3, 0.1e-3
    tip = (0.5 * L, 0.5 * L, L - needle_len)
    return dict(grid=g, L=L, v_bottom=0.0, v_top=20e5 * L, needle_length=needle_len,
                needle_radius=needle_r, seed_n0=1e19, seed_radius=1e-4, seed_center=tip,
                n_initial=1_000_000, particle_cap=20_000_000, dt=2e-12, n_ppc=75,
                w_min=1.0, growth_trigger=1.25)


# ------------------------------------------------------------------- random inputs

def rng(offset: int) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + offset)


def random_particles(n: int, g: dict | None, offset: int, vmax: float = 3e6, box=None,
                     amax: float = 0.0, w_range=(1.0, 100.0), id_base: int = 0) -> dict:
    """Particles uniform in the grid box (or `box` = (lo[3], hi[3])) with
    isotropic Gaussian velocities of scale vmax/3, weights uniform in w_range,
    ids id_base..id_base+n-1.  Values are float32-representable so that the
    FP32 and FP64 paths start from the same state."""
    r = rng(offset)
    if box is None:
        lo = np.array(g["origin"])
        hi = lo + np.array([g["nx"], g["ny"], g["nz"]]) * g["dx"]
    else:
        lo, hi = np.asarray(box[0], float), np.asarray(box[1], float)
    pos = lo + (hi - lo) * r.random((3, n)).T
    vel = r.normal(0.0, vmax / 3.0, size=(n, 3))
    acc = r.normal(0.0, amax, size=(n, 3)) if amax > 0 else np.zeros((n, 3))
    w = r.uniform(w_range[0], w_range[1], size=n)
    f = lambda a: a.astype(np.float32).astype(np.float64)
    pos = f(pos)
    # keep positions strictly inside the box after rounding to float32
    pos = np.minimum(np.maximum(pos, f(lo + 1e-9 * (hi - lo))), f(hi - 1e-6 * (hi - lo)))
    return dict(x=np.ascontiguousarray(pos[:, 0]), y=np.ascontiguousarray(pos[:, 1]),
                z=np.ascontiguousarray(pos[:, 2]),
                vx=f(vel[:, 0]), vy=f(vel[:, 1]), vz=f(vel[:, 2]),
                ax=f(acc[:, 0]), ay=f(acc[:, 1]), az=f(acc[:, 2]),
                w=f(w), id=np.arange(id_base, id_base + n, dtype=np.uint64))


def smooth_field(g: dict, offset: int, e0: float = 2e6, modes: int = 3) -> tuple:
    """A smooth random cell-centred field (V/m), float32 arrays [nz][ny][nx]."""
    r = rng(offset)
    nx, ny, nz, dx = g["nx"], g["ny"], g["nz"], g["dx"]
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny,
                          (np.arange(nx) + 0.5) / nx, indexing="ij")
    out = []
    for _ in range(3):
        f = np.full(x.shape, r.normal() * e0 * 0.5)
        for _m in range(modes):
            kx, ky, kz = r.integers(1, 4, size=3)
            ph = r.random(3) * 2 * np.pi
            f += e0 * r.normal() * np.sin(2 * np.pi * kx * x + ph[0]) * np.sin(
                2 * np.pi * ky * y + ph[1]) * np.sin(2 * np.pi * kz * z + ph[2])
        out.append(np.ascontiguousarray(f.astype(np.float32)))
    return tuple(out)


def linear_field(g: dict, grad: np.ndarray, e_at_origin: np.ndarray) -> tuple:
    """E_d(x) = e_at_origin[d] + sum_k grad[d][k] * x_k at cell centres (float32 exact
    values are not required; callers compare in float64)."""
    nx, ny, nz, dx = g["nx"], g["ny"], g["nz"], g["dx"]
    ox, oy, oz = g["origin"]
    z, y, x = np.meshgrid(oz + (np.arange(nz) + 0.5) * dx, oy + (np.arange(ny) + 0.5) * dx,
                          ox + (np.arange(nx) + 0.5) * dx, indexing="ij")
    out = []
    for d in range(3):
        f = e_at_origin[d] + grad[d][0] * x + grad[d][1] * y + grad[d][2] * z
        out.append(np.ascontiguousarray(f.astype(np.float32)))
    return tuple(out)


def random_rho(g: dict, offset: int, scale: float = 1.0) -> np.ndarray:
    """Random smooth-plus-noise charge density (C/m^3), float64 [nz][ny][nx]."""
    r = rng(offset)
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny,
                          (np.arange(nx) + 0.5) / nx, indexing="ij")
    rho = scale * (np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.4) ** 2) / 0.02)
                   + 0.1 * r.standard_normal((nz, ny, nx)))
    return np.ascontiguousarray(rho)


def swarm_en_grid(n: int = 256, lo: float = 10.0, hi: float = 1000.0) -> np.ndarray:
    """E/N values in Td, log-spaced: lo * (hi/lo)^(i/(n-1))."""
    i = np.arange(n, dtype=np.float64)
    return lo * np.power(hi / lo, i / max(n - 1, 1))


# ---------------------------------------------------------------- surrogate
MLP_SHAPES = (("W1", (128, 2)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (6, 128)),
              ("b3", (6,)))


def mlp_init(offset: int) -> np.ndarray:
    """Initial parameters of the 2-128-128-6 surrogate as one float64 vector in
    the order W1, b1, W2, b2, W3, b3 (W[o][i]): Glorot-uniform weights
    U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero biases."""
    r = rng(offset)
    parts = []
    for name, shape in MLP_SHAPES:
        if name[0] == "W":
            a = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append(r.uniform(-a, a, size=shape).ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    return np.concatenate(parts)


def mlp_query_points(n: int, offset: int, en_lo: float = 10.0, en_hi: float = 1000.0, f_lo: float = 0.1,
                     f_hi: float = 0.3) -> np.ndarray:
    """n points (E/N in Td, O2 fraction) uniform in (log10 E/N, f) over the box."""
    r = rng(offset)
    u = r.random((n, 2))
    en = 10.0 ** (np.log10(en_lo) + u[:, 0] * (np.log10(en_hi) - np.log10(en_lo)))
    f = f_lo + u[:, 1] * (f_hi - f_lo)
    return np.stack([en, f], axis=1)


# ---------------------------------------------------------------- axisymmetric
def axi_grid(nr: int, nz: int, dx: float) -> dict:
    """(r, z) mesh as a grid with one y cell and the axis at x = y = 0."""
    return grid_spec(nr, 1, nz, dx)


def needle_mask_axi(g: dict, length: float, radius: float) -> np.ndarray:
    """uint8 [nz][1][nr] mask of the ring cells whose centre (r_i, z_k) lies in a
    rod electrode on the axis hanging from the top plate, with a hemispherical
    cap whose lowest point is at z = L - length."""
    nr, nz, dx = g["nx"], g["nz"], g["dx"]
    oz = g["origin"][2]
    rc = (np.arange(nr) + 0.5) * dx
    zc = oz + (np.arange(nz) + 0.5) * dx
    zcap = oz + nz * dx - length + radius
    Z, R = np.meshgrid(zc, rc, indexing="ij")
    rod = (R <= radius) & (Z >= zcap)
    cap = (R ** 2 + (Z - zcap) ** 2) <= radius ** 2
    return np.ascontiguousarray((rod | cap).astype(np.uint8)[:, None, :])


def random_particles_axi(n: int, g: dict, offset: int, vmax: float = 3e6, w_range=(1.0, 100.0),
                         id_base: int = 0) -> dict:
    """Particles uniform in the cylinder r < nr dx, z in the grid (3D positions),
    isotropic Gaussian velocities of scale vmax/3, float32-representable."""
    r = rng(offset)
    R, L, oz = g["nx"] * g["dx"], g["nz"] * g["dx"], g["origin"][2]
    rad = R * np.sqrt(r.random(n)) * 0.999
    th = r.random(n) * 2 * np.pi
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    p = dict(x=f32(rad * np.cos(th)), y=f32(rad * np.sin(th)), z=f32(oz + L * (0.001 + 0.998 * r.random(n))))
    for k in ("vx", "vy", "vz"):
        p[k] = f32(r.normal(0, vmax / 3, n))
    for k in ("ax", "ay", "az"):
        p[k] = np.zeros(n)
    p["w"] = f32(r.uniform(*w_range, n))
    p["id"] = np.arange(id_base, id_base + n, dtype=np.uint64)
    return p


def smooth_field_axi(g: dict, offset: int, e0: float = 2e6) -> tuple:
    """A smooth random axisymmetric field on the (r, z) mesh as float32 planes
    [nz][1][nr]: (E_r, 0, E_z), with E_r vanishing on the axis."""
    r = rng(offset)
    nr, nz = g["nx"], g["nz"]
    z, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(nr) + 0.5) / nr, indexing="ij")
    er = e0 * x * (r.normal() + 0.5 * np.sin(2 * np.pi * (z + r.random())))
    ez = e0 * (r.normal() + 0.5 * np.cos(np.pi * x) * np.sin(2 * np.pi * z + r.random()))
    return (np.ascontiguousarray(er[:, None, :].astype(np.float32)), np.zeros((nz, 1, nr), np.float32),
            np.ascontiguousarray(ez[:, None, :].astype(np.float32)))
