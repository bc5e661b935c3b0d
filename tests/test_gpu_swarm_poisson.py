"""GPU swarms (Sec. 2.2.2) and multigrid Poisson (Sec. 2.5) against the CPU
oracle and closed forms, through the C ABI.

Swarm coefficients: every coefficient within 3 sigma of the oracle's (sigma
the combined batch-means errors of both runs), and within 1 % where 3 sigma is
below 1 %: the float32 swarms run at the size of the 120 Td workload (1e4
electrons, 2000 steps of 1 ps) so that 3 sigma is below 1 % for the flux drift
velocity, the mean energy, k_ion and alpha; where it is not (bulk drift,
diffusion, attachment), 3 sigma governs.  Float64 swarms follow the
oracle's trajectories exactly.  Poisson: relative residual 1e-6 and agreement
with the oracle's CG solution."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _agree(g, r, names=range(11)):
    """Coefficients outside |delta| <= 3 sigma (combined), or outside 1 % where
    3 sigma is below 1 %: (name, gpu, oracle, sigma) each."""
    bad = []
    for i in names:
        sig = np.hypot(g[11 + i], r[11 + i])
        d = abs(g[i] - r[i])
        if d > 3 * sig or (3 * sig <= 0.01 * abs(r[i]) and d > 0.01 * abs(r[i])):
            bad.append((O.RES_NAMES[i], g[i], r[i], sig))
    return bad


def _resolved_to_one_percent(g, r, names=(0, 6, 7, 9)):
    """Coefficients whose combined 3 sigma is not below 1 %: at the workload's
    size none of the flux drift velocity, the mean energy, the ionization rate
    coefficient and alpha (measured 0.07-0.54 % at 120 and 400 Td); the bulk
    drift (1.3-1.8 %), the diffusion coefficients and eta stay 3-sigma
    governed."""
    return [(O.RES_NAMES[i], 3 * np.hypot(g[11 + i], r[11 + i]) / abs(r[i])) for i in names
            if not 3 * np.hypot(g[11 + i], r[11 + i]) < 0.01 * abs(r[i])]


# the 120 Td workload's swarm size, with resampling bounds that keep the
# strongly ionizing 400 Td swarm at a few times 1e4 electrons
C1 = dict(n0=10_000, n_steps=2000, dt=1e-12, n_lo=5_000, n_hi=20_000)


def test_swarm_fp64_matches_oracle():
    from paper_2110_14494_gb300 import swarm_run
    gas = W.synthetic_air()
    seed = 2110144941
    res, mom, cnt = swarm_run(gas, [120.0], precision=64, n0=2000, n_steps=400, dt=1e-12, seed=seed,
                              n_lo=1000, n_hi=4000, want_moments=True)
    omom, ocnt, ores, _ = O.swarm(gas, 120.0, 2000, 400, 1e-12, seed, n_lo=1000, n_hi=4000)
    # same Philox streams and float64 arithmetic: the trajectories coincide
    assert np.array_equal(cnt[0], ocnt)
    scale = np.abs(omom).max(axis=0) + 1e-300
    assert np.all(np.abs(mom[0] - omom) <= 1e-9 * scale)
    assert not _agree(res[0], ores)


def _fp32_swarms_match_oracle(batched, seed):
    from paper_2110_14494_gb300 import swarm_run
    from tests.gpu_common import oracle_swarms
    ENs = (120.0, 400.0)
    res, _, _ = swarm_run(W.synthetic_air(), list(ENs), precision=32, seed=seed, batched=batched, **C1)
    ref = oracle_swarms([(EN, C1["n0"], C1["n_steps"], C1["dt"], seed + s, C1["n_lo"], C1["n_hi"])
                         for s, EN in enumerate(ENs)])
    for s, EN in enumerate(ENs):
        bad = _agree(res[s], ref[s])
        coarse = _resolved_to_one_percent(res[s], ref[s])
        rel = {O.RES_NAMES[i]: round((res[s][i] - ref[s][i]) / ref[s][i], 5) for i in range(11) if ref[s][i]}
        print(f"{'batched ' if batched else ''}float32 swarm at {EN} Td vs oracle: {rel}")
        assert not bad, (EN, bad)
        assert not coarse, (EN, coarse)


def test_swarm_fp32_matches_oracle():
    _fp32_swarms_match_oracle(False, 2110144942)


def test_swarm_constant_nu_closed_form():
    from paper_2110_14494_gb300 import swarm_run
    nu0, M = 1e12, 100 * O.M_ELEC
    gas = W.single_process_gas(W.ELASTIC, nu0 / W.N_GAS, mass=M)
    Wd = 1e5
    EN = Wd * nu0 / (O.Q_E / O.M_ELEC) / W.N_GAS / 1e-21
    for prec in (64, 32):
        res, _, _ = swarm_run(gas, [EN], precision=prec, n0=20000, n_steps=800, dt=1e-12, seed=77, kT_eV=0.5)
        assert abs(res[0][0] - Wd) / Wd < 0.02, (prec, res[0][0])
        assert abs(res[0][6] - M * Wd ** 2 / 2 / O.Q_E) / (M * Wd ** 2 / 2 / O.Q_E) < 0.03


def _centres(grid):
    nx, ny, nz, h = grid["nx"], grid["ny"], grid["nz"], grid["dx"]
    return np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                       indexing="ij")


def test_poisson_manufactured_solution():
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(64, 48, 80, 1e-4)
    h = grid["dx"]
    L = [64 * h, 48 * h, 80 * h]
    Z, Y, X = _centres(grid)
    ph = np.cos(np.pi * X / L[0]) * np.cos(np.pi * Y / L[1]) * np.sin(np.pi * Z / L[2])
    lam = sum(4 / h ** 2 * np.sin(np.pi * h / (2 * Ld)) ** 2 for Ld in L)
    rho = torch.as_tensor(O.EPS_0 * lam * ph).cuda()
    phi = torch.zeros_like(rho)
    cyc, rel = poisson_solve(grid, rho, phi, rtol=1e-10, max_cycles=60)
    assert rel <= 1e-10
    assert np.abs(phi.cpu().numpy() - ph).max() < 1e-8


def test_poisson_needle_matches_oracle_and_field():
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(32, 32, 48, 5e-5)
    L = 48 * 5e-5
    V0 = 2000.0
    mask = W.needle_mask(grid, 0.8e-3, 0.15e-3)
    rho = W.random_rho(grid, 7, 2e-2)
    ref, rr, it = O.poisson(grid, rho, mask, V0, 0.0, V0, rtol=1e-12)
    rt = torch.as_tensor(rho).cuda()
    mt = torch.as_tensor(mask).cuda()
    phi = torch.zeros_like(rt)
    E = tuple(torch.zeros(rho.shape, dtype=torch.float32, device="cuda") for _ in range(3))
    cyc, rel = poisson_solve(grid, rt, phi, mask=mt, E=E, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-10, max_cycles=100)
    assert rel <= 1e-10
    p = phi.cpu().numpy()
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-6
    Er = O.grad_phi(grid, ref, 0.0, V0)
    for a, b in zip(E, Er):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-5 * np.abs(b).max() + 1e-3
    # 1e-6 target from a cold start, with the cycle count reported
    phi2 = torch.zeros_like(rt)
    cyc2, rel2 = poisson_solve(grid, rt, phi2, mask=mt, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-6, max_cycles=100)
    assert rel2 <= 1e-6 and cyc2 < 40, (cyc2, rel2)


@pytest.mark.parametrize("prec", [64, 32])
def test_poisson_single_level_grid_matches_oracle(prec):
    """Odd sizes admit no coarser level: the whole grid (15,525 cells, more
    than one batch of the tail's loads) is the single-block tail, whose
    coarsest-level sweeps are the whole preconditioner."""
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(25, 23, 27, 5e-5)
    V0 = 1500.0
    mask = W.needle_mask(grid, 0.5e-3, 0.12e-3)
    rho = W.random_rho(grid, 13, 2e-2)
    ref, rr, it = O.poisson(grid, rho, mask, V0, 0.0, V0, rtol=1e-12)
    rt = torch.as_tensor(rho).cuda()
    mt = torch.as_tensor(mask).cuda()
    phi = torch.zeros_like(rt)
    cyc, rel = poisson_solve(grid, rt, phi, mask=mt, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-8, max_cycles=1000,
                             precision=prec)
    assert rel <= 1e-8, (cyc, rel)
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-6


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 5, 7), (6, 6, 6), (9, 7, 8), (20, 12, 36), (33, 17, 10)])
def test_poisson_shapes_match_oracle(shape, prec):
    """Edge shapes of the hierarchy: a single 2^3 level (warp-level tail
    only), odd sizes without a coarser level, x sizes that are not a multiple
    of four (the scalar stencil kernels), a tail of several levels, and a
    one-level coarsening; needle electrode where the grid holds one."""
    from paper_2110_14494_gb300 import poisson_solve
    nx, ny, nz = shape
    h = 4e-5
    grid = W.grid_spec(nx, ny, nz, h)
    V0 = 800.0
    mask = W.needle_mask(grid, 0.4 * nz * h, 1.5 * h) if min(shape) >= 6 else np.zeros((nz, ny, nx), np.uint8)
    rho = W.random_rho(grid, 3 + nx, 1e-2)
    ref, rr, it = O.poisson(grid, rho, mask, V0, 0.0, V0, rtol=1e-13)
    rt = torch.as_tensor(rho).cuda()
    mt = torch.as_tensor(mask).cuda()
    phi = torch.zeros_like(rt)
    cyc, rel = poisson_solve(grid, rt, phi, mask=mt, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-8, max_cycles=1000,
                             precision=prec)
    assert rel <= 1e-8, (cyc, rel)
    assert np.linalg.norm(phi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-6


def test_poisson_plates_only():
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(16, 16, 64, 2e-5)
    V0 = 5120.0 * 64 / 128
    rho = torch.zeros((64, 16, 16), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rho)
    E = tuple(torch.zeros((64, 16, 16), dtype=torch.float32, device="cuda") for _ in range(3))
    poisson_solve(grid, rho, phi, E=E, v_hi=V0, rtol=1e-12, max_cycles=100)
    z = (np.arange(64) + 0.5) * 2e-5
    assert np.allclose(phi.cpu().numpy(), (V0 * z / (64 * 2e-5))[:, None, None], atol=1e-7 * V0)
    assert np.allclose(E[2].cpu().numpy(), -V0 / (64 * 2e-5), rtol=1e-5)


@pytest.mark.parametrize("launch", [1, 2])
def test_batched_swarms_fp64_match_oracle_per_swarm(launch):
    """All swarms advanced together (1: the step replayed from a CUDA graph;
    2: one persistent launch for every step): each swarm's trajectory is the
    oracle's for seed + s (same counts every step, same moments)."""
    from paper_2110_14494_gb300 import swarm_run
    gas = W.synthetic_air()
    seed = 2110144950
    ENs = [60.0, 120.0, 400.0]
    res, mom, cnt = swarm_run(gas, ENs, precision=64, n0=1500, n_steps=300, dt=1e-12, seed=seed, n_lo=1000,
                              n_hi=3000, want_moments=True, batched=True, block=128, blocks_per_sm=2, use_graph=launch)
    for s, EN in enumerate(ENs):
        omom, ocnt, ores, _ = O.swarm(gas, EN, 1500, 300, 1e-12, seed + s, n_lo=1000, n_hi=3000)
        assert np.array_equal(cnt[s], ocnt), s
        scale = np.abs(omom).max(axis=0) + 1e-300
        assert np.all(np.abs(mom[s] - omom) <= 1e-9 * scale), s
        assert not _agree(res[s], ores), s


def test_batched_swarms_launch_modes_and_autotune():
    """The autotuner's choice, and the three launch modes (kernels per step, the
    step graph replayed, one persistent kernel) on the same swarms: the same
    counts every step and the moments to float rounding."""
    from paper_2110_14494_gb300 import swarm_autotune, swarm_run
    gas = W.synthetic_air()
    ENs = list(W.swarm_en_grid(16, 10.0, 1000.0))
    b, bps, chunk, mode, ms = swarm_autotune(gas, ENs, precision=32, n0=2000, n_steps=40, dt=1e-12, seed=5,
                                             n_lo=1000, n_hi=8000)
    assert b in (64, 128, 256) and bps >= 1 and chunk in (256, 512, 1024, 2048) and mode in (1, 2) and ms > 0
    kw = dict(precision=32, n0=2000, n_steps=40, dt=1e-12, seed=5, n_lo=1000, n_hi=8000, want_moments=True,
              batched=True, block=b, blocks_per_sm=bps, warp_chunk=chunk)
    runs = [swarm_run(gas, ENs, use_graph=m, **kw) for m in (0, 1, 2)]
    r1, m1, c1 = runs[1]
    for r, m, c in (runs[0], runs[2]):
        assert np.array_equal(c, c1)
        # float32 warp partial sums depend on which electrons share a flush (set
        # by the order warps take work), so the moments agree to float rounding
        scale = np.abs(m1).max(axis=1, keepdims=True) + 1e-300
        assert np.all(np.abs(m - m1) <= 1e-6 * scale)
    # resampling keeps every swarm inside its bounds (after the step that triggered it)
    assert c1.max() <= 2 * 8000 * 2 and c1[:, -1].min() > 0


@pytest.mark.parametrize("batched", [False, True])
def test_swarms_with_their_own_o2_fractions_match_oracle(batched):
    """Per-swarm O2 fractions (each swarm its own rate table and nu_max): the
    float64 trajectories are the oracle's run with that fraction's gas."""
    from paper_2110_14494_gb300 import swarm_run
    seed = 2110144970
    ENs = np.array([80.0, 150.0, 300.0, 150.0])
    fr = np.array([0.1, 0.2, 0.3, 0.25])
    res, mom, cnt = swarm_run(W.synthetic_air(), ENs, o2_frac=fr, precision=64, n0=1000, n_steps=200, dt=1e-12,
                              seed=seed, n_lo=500, n_hi=2500, want_moments=True, batched=batched,
                              block=128 if batched else 0, blocks_per_sm=2 if batched else 0)
    for s in range(len(ENs)):
        omom, ocnt, ores, _ = O.swarm(W.synthetic_air(o2_frac=fr[s]), ENs[s], 1000, 200, 1e-12, seed + s,
                                      n_lo=500, n_hi=2500)
        assert np.array_equal(cnt[s], ocnt), s
        scale = np.abs(omom).max(axis=0) + 1e-300
        assert np.all(np.abs(mom[s] - omom) <= 1e-9 * scale), s


def test_o2_fractions_need_tagged_species():
    from paper_2110_14494_gb300 import PicError, swarm_run
    gas = W.synthetic_air()
    del gas["species"]
    with pytest.raises(PicError) as e:
        swarm_run(gas, [100.0], o2_frac=[0.2], n0=100, n_steps=30, n_lo=10, n_hi=400)
    assert e.value.code == -1


def test_batched_swarms_fp32_match_oracle():
    _fp32_swarms_match_oracle(True, 2110144960)


def test_poisson_pair_precision_matches_oracle():
    """Float-pair potential, float32 CG with refinement (precision 32): the
    needle problem from a cold start (several refinement passes) against the
    oracle's float64 CG solution."""
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(32, 32, 48, 5e-5)
    V0 = 2000.0
    mask = W.needle_mask(grid, 0.8e-3, 0.15e-3)
    rho = W.random_rho(grid, 7, 2e-2)
    ref, rr, it = O.poisson(grid, rho, mask, V0, 0.0, V0, rtol=1e-12)
    rt = torch.as_tensor(rho).cuda()
    mt = torch.as_tensor(mask).cuda()
    phi = torch.zeros_like(rt)
    E = tuple(torch.zeros(rho.shape, dtype=torch.float32, device="cuda") for _ in range(3))
    cyc, rel = poisson_solve(grid, rt, phi, mask=mt, E=E, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-8, max_cycles=100,
                             precision=32)
    assert rel <= 1e-8 and cyc < 40, (cyc, rel)
    p = phi.cpu().numpy()
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-5
    assert np.all(p[mask != 0] == V0)
    Er = O.grad_phi(grid, ref, 0.0, V0)
    for a, b in zip(E, Er):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-5 * np.abs(b).max() + 1e-3


def test_poisson_pair_precision_plates_and_warm_start():
    """Plates only: the linear potential to float-pair accuracy; a warm start
    at the solution needs no iteration."""
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(16, 16, 64, 2e-5)
    V0 = 2560.0
    rho = torch.zeros((64, 16, 16), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rho)
    E = tuple(torch.zeros((64, 16, 16), dtype=torch.float32, device="cuda") for _ in range(3))
    poisson_solve(grid, rho, phi, E=E, v_hi=V0, rtol=1e-8, max_cycles=100, precision=32)
    z = (np.arange(64) + 0.5) * 2e-5
    exact = (V0 * z / (64 * 2e-5))[:, None, None]
    assert np.abs(phi.cpu().numpy() - exact).max() < 1e-6 * V0
    assert np.allclose(E[2].cpu().numpy(), -V0 / (64 * 2e-5), rtol=1e-5)
    phi2 = torch.as_tensor(np.broadcast_to(exact, (64, 16, 16)).copy()).cuda()
    cyc, rel = poisson_solve(grid, rho, phi2, v_hi=V0, rtol=1e-8, max_cycles=100, precision=32)
    assert cyc == 0 and rel <= 1e-8, (cyc, rel)


def test_poisson_pair_precision_agrees_with_float64_solve():
    """The two precisions of the GPU solve on a 64^3 needle with a streamer-like
    charge: solutions within the tolerance they were solved to."""
    from paper_2110_14494_gb300 import poisson_solve
    grid = W.grid_spec(64, 64, 64, 4e-5)
    L = 64 * 4e-5
    V0 = 20e5 * L
    mask = torch.as_tensor(W.needle_mask(grid, 1.0e-3, 0.2e-3)).cuda()
    rho = torch.as_tensor(W.random_rho(grid, 11, 5e-2)).cuda()
    out = []
    for prec in (64, 32):
        phi = torch.zeros_like(rho)
        cyc, rel = poisson_solve(grid, rho, phi, mask=mask, v_lo=0.0, v_hi=V0, v_mask=V0, rtol=1e-8,
                                 max_cycles=100, precision=prec)
        assert rel <= 1e-8
        out.append(phi.cpu().numpy())
    assert np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[0]) < 1e-6
