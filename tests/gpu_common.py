"""Helpers shared by the GPU tests (comparison of particle sets)."""
import numpy as np


def by_id(p: dict) -> dict:
    o = np.argsort(p["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in p.items()}


def compare_sets(gpu: dict, ref: dict, dx: float, rtol: float, v_floor: float = 1e4):
    """Returns (n_common, n_only_gpu, n_only_ref, n_bad, worst) where n_bad
    counts common particles outside the tolerance:
    |dx| / dx_cell <= rtol and |dv| / (|v| + v_floor) <= rtol and |dw| <= rtol w."""
    g, r = by_id(gpu), by_id(ref)
    common, ig, ir = np.intersect1d(g["id"], r["id"], assume_unique=True, return_indices=True)
    pos = max(np.abs(g[k][ig] - r[k][ir]).max(initial=0) for k in ("x", "y", "z"))
    perr = np.max([np.abs(g[k][ig] - r[k][ir]) / dx for k in ("x", "y", "z")], axis=0) if len(common) else np.zeros(0)
    sp = np.sqrt(r["vx"][ir] ** 2 + r["vy"][ir] ** 2 + r["vz"][ir] ** 2) + v_floor
    verr = np.max([np.abs(g[k][ig] - r[k][ir]) / sp for k in ("vx", "vy", "vz")], axis=0) if len(common) else \
        np.zeros(0)
    werr = np.abs(g["w"][ig] - r["w"][ir]) / np.maximum(np.abs(r["w"][ir]), 1e-300) if len(common) else np.zeros(0)
    err = np.maximum(np.maximum(perr, verr), werr) if len(common) else np.zeros(0)
    bad = err > rtol
    worst = dict(pos=float(perr.max(initial=0)), vel=float(verr.max(initial=0)), w=float(werr.max(initial=0)),
                 abs_pos=float(pos), gross=int((err > 1e-3).sum()))
    return len(common), len(g["id"]) - len(common), len(r["id"]) - len(common), int(bad.sum()), worst


def rel_energy_error(gpu: dict, ref: dict, q: float) -> float:
    """The q-quantile over the common particles of |eps_gpu - eps_ref| / eps_ref."""
    g, r = by_id(gpu), by_id(ref)
    _, ig, ir = np.intersect1d(g["id"], r["id"], assume_unique=True, return_indices=True)
    eg = g["vx"][ig] ** 2 + g["vy"][ig] ** 2 + g["vz"][ig] ** 2
    er = r["vx"][ir] ** 2 + r["vy"][ir] ** 2 + r["vz"][ir] ** 2
    ok = er > 0
    return float(np.quantile(np.abs(eg[ok] - er[ok]) / er[ok], q)) if ok.any() else 0.0


def ill_conditioned(advance, before: dict, capacity: int, ref: dict, dx: float, tol: float, delta: float,
                    seed: int):
    """The oracle's own conditioning: the same starting state with every
    energy moved by delta (relative, random sign) is advanced by
    advance(particles) and compared with the unperturbed result ref.
    Returns (flips: gross differences and particles on one side only, the
    other particles outside tol).  Decisions taken within delta of their
    thresholds flip, and near an inelastic threshold eps - eps_th amplifies
    the error by eps / (eps - eps_th), whatever its source."""
    import oracle as O
    r = np.random.default_rng(seed)
    s = np.sqrt(1.0 + delta * r.choice([-1.0, 1.0], size=len(before["vx"])))
    pert = {k: (np.asarray(v) * s if k in ("vx", "vy", "vz") else np.array(v, copy=True)) for k, v in before.items()}
    P = O.Particles(capacity, pert)
    advance(P)
    _, og, orf, bad, worst = compare_sets(P.view(), ref, dx, tol, v_floor=1e5)
    return worst["gross"] + og + orf, bad - worst["gross"]


def oracle_swarm_results(job):
    """The oracle's swarm coefficients for one (E/N, seed) job; a top-level
    function so that spawned worker processes can run several at once."""
    import oracle as O
    import workloads as W
    EN, n0, n_steps, dt, seed, n_lo, n_hi = job
    return O.swarm(W.synthetic_air(), EN, n0, n_steps, dt, seed, n_lo=n_lo, n_hi=n_hi)[2]


def oracle_swarms(jobs):
    """Runs oracle swarms in parallel in spawned processes (no CUDA state is
    inherited); returns their coefficient vectors in job order."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(oracle_swarm_results, jobs))
