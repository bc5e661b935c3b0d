"""The float32 coupled field solve driven on the device (one CUDA graph per
solve whose conditional nodes run the flexible-CG loop, Sec. 2.5) against
the same solve driven from the host: identical decisions on identical values,
so the particle sets, the potentials and the reported cycles and residuals
agree bit for bit; the cycle limit is still reported."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import by_id

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 2110144940


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _streamer_ctx(device_loop, rtol=1e-6, grid_n=32, growth_trigger=1.5):
    """A small needle-plane streamer: a Gaussian seed below a charged needle,
    coupled float32 solve, weight updates on growth."""
    from paper_2110_14494_gb300 import PicContext
    grid = W.grid_spec(grid_n, grid_n, grid_n + 16, 2.5e-5)
    mask = W.needle_mask(grid, 0.35e-3, 0.08e-3)
    V0 = 4000.0
    ctx = PicContext(W.synthetic_air(), grid, precision=32, capacity=400_000, seed=SEED, dt=2e-12, mask=mask,
                     coupled=True, v_lo=0.0, v_hi=V0, v_mask=V0, poisson_rtol=rtol, poisson_max_cycles=60,
                     boundary=1, growth_trigger=growth_trigger, particle_cap=150_000)
    ctx.set_poisson(rtol, 60, device_loop=device_loop)
    L = grid_n * 2.5e-5
    ctx.seed_gaussian(5e19, 6e-5, (0.5 * L, 0.5 * L, 0.45 * (grid_n + 16) * 2.5e-5), 2e3)
    return ctx


def _phi(ctx, n):
    blob = ctx.save()
    return np.frombuffer(blob, np.float64, count=n, offset=len(blob) - 8 * n).copy()


def test_device_loop_matches_host_loop():
    n = 32 * 32 * 48
    a = _streamer_ctx(True)
    b = _streamer_ctx(False)
    for step in range(8):
        sa = a.step(1, stats=True)
        sb = b.step(1, stats=True)
        assert sa.poisson_cycles == sb.poisson_cycles, step
        assert sa.poisson_rel_res == sb.poisson_rel_res, step
        assert sa.poisson_rel_res <= 1e-6
        assert sa.n_end == sb.n_end, step
    assert np.array_equal(_phi(a, n), _phi(b, n))
    pa, pb = by_id(a.get_particles()), by_id(b.get_particles())
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


def test_device_loop_reports_cycle_limit():
    from paper_2110_14494_gb300 import PicError
    for device_loop in (True, False):
        ctx = _streamer_ctx(device_loop)
        ctx.step(3)                      # the third solve already runs as a graph on the device loop
        ctx.set_poisson(1e-14, 1, device_loop=device_loop)   # unreachable: the float pair bounds it near 1e-9
        with pytest.raises(PicError) as ei:
            ctx.step(2)
        assert "cycle limit" in str(ei.value)


def test_device_loop_counts_its_kernels():
    # no weight updates: every speculative solve stands
    a = _streamer_ctx(True, growth_trigger=0.0)
    b = _streamer_ctx(False, growth_trigger=0.0)
    for c in (a, b):
        c.step(2)
        c.profile(True)
        c.step(4)
    pa, pb = a.profile(False), b.profile(False)
    assert pa["n_speculative"] == 4 and pa["n_undone"] == 0
    assert pb["n_speculative"] == 0
    # the same work; per solve the device-driven graph adds its gate, the
    # priming and checking kernels of the loop, one decision kernel per loop
    # trip and one report kernel, and counts its branches' kernels on the
    # device
    assert pb["n_launches"] > 0
    assert pb["n_launches"] < pa["n_launches"] <= pb["n_launches"] + 4 * 12


def _axi_ctx(device_loop, prec=64):
    """A small axisymmetric needle-plane run (ring cells, float64 multigrid CG)."""
    from paper_2110_14494_gb300 import PicContext
    g = W.axi_grid(64, 128, 2e-5)
    L, V = 128 * 2e-5, 20e5 * 128 * 2e-5
    mk = W.needle_mask_axi(g, 0.5e-3, 0.1e-3)
    ctx = PicContext(W.synthetic_air(), g, precision=prec, geometry=1, capacity=1_000_000, seed=SEED, dt=2e-12,
                     mask=mk, coupled=True, v_lo=0.0, v_hi=V, v_mask=V, poisson_rtol=1e-8, poisson_max_cycles=80,
                     boundary=1)
    ctx.set_poisson(1e-8, 80, device_loop=device_loop)
    ctx.seed_gaussian(1e19, 1e-4, (0.0, 0.0, L - 0.5e-3), 100.0)
    return ctx


def test_axi_device_loop_matches_host_loop():
    """The axisymmetric solve adds its block sums with atomics, so the two
    drivers agree to rounding, not bit for bit: the same cycle counts, the
    residuals within 1e-3 of each other, and float64 particles within 1e-9
    after six coupled steps."""
    a, b = _axi_ctx(True), _axi_ctx(False)
    for step in range(6):
        sa, sb = a.step(1, stats=True), b.step(1, stats=True)
        assert sa.poisson_cycles == sb.poisson_cycles, step
        assert sa.poisson_rel_res <= 1e-8 and sb.poisson_rel_res <= 1e-8
        assert abs(sa.poisson_rel_res - sb.poisson_rel_res) <= 1e-3 * sb.poisson_rel_res + 1e-14
        assert sa.n_end == sb.n_end, step
    pa, pb = by_id(a.get_particles()), by_id(b.get_particles())
    assert np.array_equal(pa["id"], pb["id"])
    for k in ("x", "y", "z"):
        assert np.abs(pa[k] - pb[k]).max() <= 1e-9 * 128 * 2e-5, k
    for k in ("vx", "vy", "vz"):
        assert np.abs(pa[k] - pb[k]).max() <= 1e-9 * (np.abs(pb[k]).max() + 1e5), k


def test_axi_device_loop_reports_cycle_limit():
    from paper_2110_14494_gb300 import PicError
    ctx = _axi_ctx(True)
    ctx.step(3)
    ctx.set_poisson(1e-15, 1, device_loop=True)
    with pytest.raises(PicError) as ei:
        ctx.step(2)
    assert "cycle limit" in str(ei.value)


def test_device_loop_refinement_branch_matches_host_loop():
    """At rtol 1e-9 the float32 correction must be committed and the pair
    residual re-formed (iterative refinement) within a solve: the device
    loop's refinement branch against the host loop, bit for bit."""
    n = 32 * 32 * 48
    a = _streamer_ctx(True, rtol=1e-9)
    b = _streamer_ctx(False, rtol=1e-9)
    for step in range(5):
        sa = a.step(1, stats=True)
        sb = b.step(1, stats=True)
        assert sa.poisson_cycles == sb.poisson_cycles, step
        assert sa.poisson_rel_res == sb.poisson_rel_res, step
        assert sa.poisson_rel_res <= 1e-9
    assert np.array_equal(_phi(a, n), _phi(b, n))
    pa, pb = by_id(a.get_particles()), by_id(b.get_particles())
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


@pytest.mark.parametrize("photo", [False, True])
def test_speculative_solve_is_undone_exactly(photo):
    """The device-driven solve of a step is enqueued before the host has read
    the step's counts; a step whose counts then call for a weight update (the
    particles grew) or for further product generations (cascades deeper than
    a lane's stack) undoes it and solves again after them.  Ionization at
    2e12/s (four per electron per 2 ps step, so cascades overflow the lane
    stacks) against attachment at 1.9e12/s (net growth e^0.2 per step, so the
    fixed-point deposit stays far from overflow) and a growth trigger of 1.01
    make both happen in most steps: particle sets, potentials, cycle counts
    and residuals equal those of the host-driven run, which never
    speculates, bit for bit."""
    from paper_2110_14494_gb300 import PicContext
    from paper_2110_14494_gb300 import picmcc as P
    gas = W.multi_gas([W.single_process_gas(W.ELASTIC, 1e12 / W.N_GAS, mass=0.0),
                       W.single_process_gas(W.IONIZATION, 2e12 / W.N_GAS, threshold=0.0),
                       W.single_process_gas(W.ATTACHMENT, 1.9e12 / W.N_GAS)])
    grid = W.grid_spec(32, 32, 48, 2.5e-5)
    mask = W.needle_mask(grid, 0.35e-3, 0.08e-3)
    V0 = 4000.0
    kw = {}
    if photo:
        pq, p = 4000.0, 101325.0
        kw = dict(photo_xi=0.05 * (p + pq) / pq, photo_pq=pq, pressure=p, p_o2=0.2 * p,
                  chi_min=P.ZHELEZNYAK_CHI_MIN, chi_max=P.ZHELEZNYAK_CHI_MAX)

    def ctx_(device_loop):
        c = PicContext(gas, grid, precision=32, capacity=600_000, seed=SEED, dt=2e-12, mask=mask, coupled=True,
                       v_lo=0.0, v_hi=V0, v_mask=V0, poisson_rtol=1e-6, poisson_max_cycles=80, boundary=1,
                       growth_trigger=1.01, particle_cap=4000, **kw)
        c.set_poisson(1e-6, 80, device_loop=device_loop)
        L = 32 * 2.5e-5
        c.seed_gaussian(5e17, 6e-5, (0.5 * L, 0.5 * L, 0.45 * 48 * 2.5e-5), 200.0)
        return c

    n = 32 * 32 * 48
    a, b = ctx_(True), ctx_(False)
    a.profile(True)
    wu = 0
    for step in range(6):
        sa = a.step(1, stats=True)
        sb = b.step(1, stats=True)
        assert sa.n_end == sb.n_end, step
        assert sa.n_children == sb.n_children, step
        assert sa.poisson_cycles == sb.poisson_cycles, step
        assert sa.poisson_rel_res == sb.poisson_rel_res, step
        assert sa.n_weight_updates == sb.n_weight_updates, step
        wu += sa.n_weight_updates
    assert wu >= 3
    pa = a.profile(False)
    assert pa["n_speculative"] >= 4 and pa["n_undone"] >= 3, pa
    assert np.array_equal(_phi(a, n), _phi(b, n))
    pa, pb = by_id(a.get_particles()), by_id(b.get_particles())
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
