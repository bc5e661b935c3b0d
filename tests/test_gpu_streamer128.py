"""Oracle parity on the benchmarked workload: the coupled 128^3 streamer
(Sec. 2.1 step, Sec. 2.3 geometry and seed, Sec. 2.5 space charge and
Poisson), built by the benchmark's own context factory (same launch shapes,
weight-update trigger, sort interval, adaptive time step, outflow faces).

At steps 1, 10 and 100 the GPU's particle state before the step and the field
its gather reads are downloaded, and the oracle advances that state through
the same step (same step index, dt, half-kick length, field, electrode).
Compared:
- particles: float64 1e-12 per particle; float32 1e-5 (position per cell,
  velocity per |v| + 1e5 m/s) with decision flips (gross differences and
  particles on one side only) at most 1e-5 N + 2, and the other particles
  outside 1e-5 (rounding amplification near inelastic thresholds: eps -
  eps_th carries the error of eps times eps / (eps - eps_th)) at most twice
  the step's own conditioning plus 10: the count the oracle leaves outside
  1e-5 when it advances the same state with every energy moved by the
  float32 path's measured error (the 90th percentile of |d eps| / eps over
  the common particles, 1.4-1.9e-6); measured 843 and 987 particles against
  1133 and 2375 at steps 11 and 100, ending the step with a median energy of
  0.7-1.6 eV against 5 eV for all;
- the deposit the step's own kernels made (pic_get_deposit) against the
  oracle's deposit of the GPU's particles after the step: bit for bit;
- the ion grids' increments over the step against the oracle's (the same
  events up to the flips);
- the space charge of pic_deposit against the oracle's fixed-to-rho of the
  same grids;
- the potential the coupled solve made from that charge (float pairs in
  float32, float64 CG in float64): its residual under the oracle's operator
  within the solve's tolerance, and, at step 10, its distance to the oracle's
  CG solution of the same system; the field for the next step against the
  oracle's gradient of that solution.
A step that ran a weight update is skipped for the next one (merged
particles cannot be compared with the oracle's unmerged step)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_common import compare_sets, ill_conditioned, rel_energy_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 2110144940


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _np(t):
    return t.detach().cpu().numpy()


def _field(ctx):
    return tuple(np.ascontiguousarray(_np(f)) for f in ctx.get_field())


def _grids(ctx, n, fresh=False):
    q = [torch.zeros(n, dtype=torch.int64, device="cuda") for _ in range(3)]
    (ctx.deposit if fresh else ctx.get_deposit)(*q)
    return [_np(a) for a in q]


def _energy_split(gpu, ref, dx, tol):
    """Median final kinetic energy (eV, oracle) of all common particles and of
    those outside tol but not gross (position per cell, velocity per |v| +
    1e5 m/s; gross: beyond 1e-3, the decision flips counted separately)."""
    from tests.gpu_common import by_id
    G, R = by_id(gpu), by_id(ref)
    common, ig, ir = np.intersect1d(G["id"], R["id"], assume_unique=True, return_indices=True)
    sp = np.sqrt(R["vx"][ir] ** 2 + R["vy"][ir] ** 2 + R["vz"][ir] ** 2)
    err = np.max([np.abs(G[k][ig] - R[k][ir]) / dx for k in ("x", "y", "z")] +
                 [np.abs(G[k][ig] - R[k][ir]) / (sp + 1e5) for k in ("vx", "vy", "vz")], axis=0)
    e = 0.5 * O.M_ELEC * sp ** 2 / O.Q_E
    out = (err > tol) & (err <= 1e-3)
    return float(np.median(e)), float(np.median(e[out])) if out.any() else 0.0


def _phi(ctx, n):
    blob = ctx.save()
    return np.frombuffer(blob, np.float64, count=n, offset=len(blob) - 8 * n).copy()


@pytest.mark.parametrize("prec", [32, 64])
def test_coupled_streamer_128_matches_oracle(prec):
    import bench
    wl = bench.workload(128, 1_000_000)
    g = wl["grid"]
    n = g["nx"] * g["ny"] * g["nz"]
    dV = g["dx"] ** 3
    V = wl["v_top"]
    mask = W.needle_mask(g, wl["needle_length"], wl["needle_radius"])
    gas = W.synthetic_air()
    ctx = bench.streamer_context(wl, prec, capacity=6_000_000, seed=SEED)
    ctx.seed_gaussian(wl["seed_n0"], wl["seed_radius"], wl["seed_center"], bench.seed_weight(wl))
    ctx.step(0)  # the first field, from the neutral seed
    dt_prev, done = 0.0, 0
    checks = (1, 10, 100) if prec == 32 else (1, 10)
    tol = 1e-5 if prec == 32 else 1e-12
    for k in checks:
        if k - 1 > done:
            st = ctx.step(k - 1 - done, stats=True)
            dt_prev, done = st.dt_last, k - 1
        while True:
            before = ctx.get_particles()
            field = _field(ctx)
            qp0, qn0 = _grids(ctx, n)[1:]
            st = ctx.step(1, stats=True)
            done += 1
            if st.n_weight_updates == 0:
                break
            dt_prev = st.dt_last
        gpu = ctx.get_particles()
        q_step = _grids(ctx, n)
        phi = _phi(ctx, n)
        next_field = _field(ctx)
        q_fresh = _grids(ctx, n, fresh=True)
        rho_t = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.deposit(rho=rho_t)
        rho_gpu = _np(rho_t)

        # the oracle advances the GPU's state through the same step
        m = O.Model(gas, st.dt_last, SEED, 64, g, field, mask=mask, boundary=1, dt_kick=dt_prev)
        P = O.Particles(3 * len(before["x"]) + 1024, before)
        rq_e = np.zeros(n, np.int64)
        rq_pos, rq_neg = qp0.copy(), qn0.copy()
        rc, ost = O.step(m, P, done, done == 1, rq_e, rq_pos, rq_neg)
        assert rc == 0
        ref = P.view()
        N = len(ref["id"])
        nc, og, orf, bad, worst = compare_sets(gpu, ref, g["dx"], tol, v_floor=1e5 if prec == 32 else 1.0)
        flips = worst["gross"] + og + orf
        print(f"step {done} prec {prec}: N {N} common {nc} only-gpu {og} only-oracle {orf} "
              f"outside {tol:g}: {bad} {worst}")
        if prec == 64:
            assert og == 0 and orf == 0 and bad == 0, (done, og, orf, bad, worst)
        else:
            assert flips <= 1e-5 * N + 2, (done, flips, worst)
            # rounding amplification: bounded by the step's own conditioning under the float32 path's
            # measured energy error (its 90th percentile over the common particles)
            delta = rel_energy_error(gpu, ref, 0.9)

            def advance(Pp):
                rc, _ = O.step(m, Pp, done, done == 1, np.zeros(n, np.int64), qp0.copy(), qn0.copy())
                assert rc == 0
            c_flips, c_bad = ill_conditioned(advance, before, 3 * len(before["x"]) + 1024, ref, g["dx"], tol, delta,
                                             1000 + done)
            print(f"step {done}: energy error 90th percentile {delta:.3g}; under it the oracle has {c_flips} flips "
                  f"and {c_bad} more outside {tol:g}; float32: {flips} flips, {bad - worst['gross']} more")
            assert bad - worst["gross"] <= 2 * c_bad + 10, (done, bad, worst, c_bad, delta)
            # the particles outside 1e-5 are the rounding amplification of an inelastic loss (eps - eps_th
            # carries the float32 error of eps times eps / (eps - eps_th)): they end the step slow
            e_med, e_bad = _energy_split(gpu, ref, g["dx"], tol)
            print(f"step {done}: median final energy {e_med:.3g} eV, of the particles outside {tol:g} {e_bad:.3g} eV")
            assert bad - worst["gross"] == 0 or e_bad < 0.5 * e_med, (done, e_bad, e_med)
        assert abs(st.n_events - ost.n_events) <= 1e-4 * ost.n_events + 10

        # the step's own deposit is the deposit of the particles it left, bit for bit
        m_dep = O.Model(gas, st.dt_last, SEED, prec, g)
        q_ref = O.deposit(m_dep, O.Particles(len(gpu["x"]), gpu))
        assert np.array_equal(q_step[0], q_ref), done
        assert np.array_equal(q_fresh[0], q_ref), done
        assert np.array_equal(q_fresh[1], q_step[1]) and np.array_equal(q_fresh[2], q_step[2])
        # ion events of the step: each adds exactly llrint(w 2^32) to its grid's total
        for a, b, q0 in ((q_step[1], rq_pos, qp0), (q_step[2], rq_neg, qn0)):
            dg, dr = int((a - q0).sum()), int((b - q0).sum())
            wmax = float(before["w"].max()) * 2.0 ** 32
            assert abs(dg - dr) <= flips * wmax + 64, (done, dg, dr)
            if prec == 64:
                assert np.abs((a - q0) - (b - q0)).max() <= 64, done

        # space charge of the GPU's grids, then the potential the coupled solve made from it
        rho_ref = O.fixed_to_rho(dV, q_step[0], q_step[1], q_step[2])
        assert np.allclose(rho_gpu, rho_ref, rtol=1e-12, atol=1e-12 * np.abs(rho_ref).max()), done
        assert np.abs(rho_ref).max() > 0.0
        _, rel, _ = O.poisson(g, rho_ref.reshape(g["nz"], g["ny"], g["nx"]), mask, V, 0.0, V, max_iter=0,
                              phi0=phi)
        assert rel <= 1.5e-6, (done, rel)
        assert np.all(phi.reshape(mask.shape)[mask > 0] == V)
        # the field is the central-difference gradient of that potential: the oracle's gradient of the
        # GPU's own potential, to the float32 rounding of the field (float64 contexts: float64 rounding)
        Eg = O.grad_phi(g, phi.reshape(g["nz"], g["ny"], g["nx"]), 0.0, V)
        emax = max(np.abs(e).max() for e in Eg)
        gtol = 2e-6 if prec == 32 else 1e-12
        for a, b in zip(next_field, Eg):
            assert np.abs(a.ravel() - b.ravel()).max() <= gtol * emax, (done, np.abs(a.ravel() - b.ravel()).max() / emax)
        if k == 10:
            phi_ref, rel_ref, _ = O.poisson(g, rho_ref.reshape(g["nz"], g["ny"], g["nx"]), mask, V, 0.0, V,
                                            rtol=1e-10)
            d = np.linalg.norm(phi - phi_ref.ravel()) / np.linalg.norm(phi_ref)
            Er = O.grad_phi(g, phi_ref, 0.0, V)
            de = max(np.abs(a.ravel() - b.ravel()).max() for a, b in zip(next_field, Er)) / emax
            print(f"step {done}: potential vs the oracle's CG {d:.2e}, field {de:.2e} of max |E| "
                  f"(solve residual {rel:.2e})")
            # a residual of 1e-6 leaves an error whose central differences reach ~1e-4 of the peak field at the
            # needle tip (measured 1.0e-4 at step 11); the bound is the solve tolerance's, not the gradient's
            assert d <= 1e-5, d
            assert de <= 5e-4, de
        dt_prev = st.dt_last
