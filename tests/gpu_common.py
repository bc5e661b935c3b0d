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
