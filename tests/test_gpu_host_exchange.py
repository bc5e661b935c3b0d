"""Native-precision particle exchange with host memory (pic_upload,
pic_download): exact round trips, the same steps as the double-precision
exchange (pic_set_particles / pic_get_particles), and the capacity error."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import by_id

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 2110144940
GRID = W.grid_spec(24, 20, 28, 2e-5, origin=(1e-5, -2e-5, 0.0))
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "w")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def _ctx(prec, cap):
    from paper_2110_14494_gb300 import PicContext
    return PicContext(W.synthetic_air(), GRID, precision=prec, capacity=cap, seed=SEED, dt=2e-12)


def _native(p, prec, cap):
    """11 host arrays of capacity cap in the context precision (ids int64)."""
    dt = np.float32 if prec == 32 else np.float64
    arrs = [np.zeros(cap, dt) for _ in FIELDS] + [np.zeros(cap, np.int64)]
    n = len(p["x"])
    for a, k in zip(arrs, FIELDS):
        a[:n] = p[k]
    arrs[10][:n] = p["id"].astype(np.int64)
    return arrs


def _native_block(p, prec, cap):
    """The same 11 arrays with the ten real ones as rows of one host block
    (one pitched copy each way)."""
    dt = np.float32 if prec == 32 else np.float64
    block = np.zeros((10, cap), dt)
    arrs = [block[i] for i in range(10)] + [np.zeros(cap, np.int64)]
    n = len(p["x"])
    for a, k in zip(arrs, FIELDS):
        a[:n] = p[k]
    arrs[10][:n] = p["id"].astype(np.int64)
    return arrs


def _as_dict(arrs, n):
    d = {k: arrs[i][:n].astype(np.float64) for i, k in enumerate(FIELDS)}
    d["id"] = arrs[10][:n].astype(np.uint64)
    return d


@pytest.mark.parametrize("prec,block", [(32, False), (64, False), (32, True), (64, True)])
def test_upload_download_round_trip_is_exact(prec, block):
    """Separate host arrays (eleven copies each way) and the real arrays as
    rows of one host block (a pitched copy), in and out in both layouts."""
    p0 = W.random_particles(5000, GRID, 17, vmax=2e6, w_range=(1.0, 9.0))
    cap = 8000
    ctx = _ctx(prec, cap)
    up = (_native_block if block else _native)(p0, prec, cap)
    ctx.upload(up, 5000, accel_valid=True)
    for back in ([np.zeros_like(a) for a in up], _native_block({k: np.zeros(0) for k in FIELDS + ("id",)}, prec,
                                                               cap)):
        n = ctx.download(back, cap)
        assert n == 5000
        for a, b in zip(up, back):
            assert np.array_equal(a[:n], b[:n])
    # the same through host sets checked once
    hs_up, back = ctx.host_set(up, cap), [np.zeros_like(a) for a in up]
    hs_back = ctx.host_set(back, cap)
    ctx.upload(hs_up, 5000, accel_valid=True)
    assert ctx.download(hs_back) == 5000
    for a, b in zip(up, back):
        assert np.array_equal(a[:5000], b[:5000])
    # the double-precision read-back sees the same particles
    g = by_id(ctx.get_particles())
    ref = by_id(_as_dict(up, n))
    for k in ref:
        assert np.array_equal(g[k], ref[k]), k


@pytest.mark.parametrize("prec", [32, 64])
def test_steps_through_host_buffers_match_resident_steps(prec):
    """Three steps with the particles resident against three steps each
    uploaded from and downloaded to host buffers: the same particles, bit for
    bit (the first without a half-kick in both, the others with the uploaded
    accelerations)."""
    p0 = W.random_particles(4000, GRID, 29, vmax=3e6, w_range=(1.0, 500.0))
    F = W.smooth_field(GRID, 131, e0=3e6)
    Fd = tuple(torch.as_tensor(f).cuda() for f in F)
    cap = 40000
    a = _ctx(prec, cap)
    a.set_field(*Fd)
    a.set_particles(p0)
    a.step(3)
    ra = by_id(a.get_particles())

    b = _ctx(prec, cap)
    b.set_field(*Fd)
    dt = np.float32 if prec == 32 else np.float64
    q = {k: p0[k].astype(dt) for k in FIELDS}
    q["id"] = p0["id"]
    host = _native(q, prec, cap)
    n = 4000
    for s in range(3):
        b.upload(host, n, accel_valid=s > 0)
        b.step(1)
        n = b.download(host, cap)
    rb = by_id(_as_dict(host, n))
    assert np.array_equal(ra["id"], rb["id"])
    for k in FIELDS:
        assert np.array_equal(ra[k], rb[k]), k


def test_download_into_too_small_arrays_is_reported():
    from paper_2110_14494_gb300 import PicError
    p0 = W.random_particles(3000, GRID, 5)
    ctx = _ctx(32, 8000)
    ctx.set_particles(p0)
    small = [np.zeros(1000, np.float32) for _ in FIELDS] + [np.zeros(1000, np.int64)]
    with pytest.raises(PicError):
        ctx.download(small, 1000)


def _coupled_streamer():
    """A small coupled float32 needle-plane streamer (speculative field
    solves from the third step on, weight updates on growth)."""
    from paper_2110_14494_gb300 import PicContext
    grid = W.grid_spec(32, 32, 48, 2.5e-5)
    mask = W.needle_mask(grid, 0.35e-3, 0.08e-3)
    V0 = 4000.0
    ctx = PicContext(W.synthetic_air(), grid, precision=32, capacity=400_000, seed=SEED, dt=2e-12, mask=mask,
                     coupled=True, v_lo=0.0, v_hi=V0, v_mask=V0, poisson_rtol=1e-6, poisson_max_cycles=60,
                     boundary=1, growth_trigger=1.5, particle_cap=150_000)
    L = 32 * 2.5e-5
    ctx.seed_gaussian(5e19, 6e-5, (0.5 * L, 0.5 * L, 0.45 * 48 * 2.5e-5), 2e3)
    return ctx


def test_exchanges_under_the_speculative_solve_match_ordered_ones():
    """Steps through pinned host buffers (download, then upload, after every
    step): right after a speculative step both copies overlap the solve on
    the exchange stream; a context that makes one other call first (pic_count)
    exchanges on its own stream behind the solve.  Bit-identical particle sets
    every step, and the overlapped exchanges are counted."""
    cap = 400_000
    ctxs, hosts = [], []
    for _ in range(2):
        ctx = _coupled_streamer()
        block = torch.empty((10, cap), dtype=torch.float32, pin_memory=True)
        ids = torch.empty(cap, dtype=torch.int64, pin_memory=True)
        hs = ctx.host_set([block[i] for i in range(10)] + [ids], cap)
        ctx.profile(True)
        ctxs.append(ctx)
        hosts.append((hs, block, ids))
    a, b = ctxs
    (ha, ba, ia), (hb, bb, ib) = hosts

    def sets(block, ids, n):  # the particle set by id (the output order of the collision kernel varies)
        return by_id(_as_dict([block[i].numpy() for i in range(10)] + [ids.numpy()], n))

    for step in range(12):
        a.step(1)
        b.step(1)
        b.count()                 # any call in between: the exchanges then wait for the solve
        na = a.download(ha)
        nb = b.download(hb)
        assert na == nb, step
        sa, sb = sets(ba, ia, na), sets(bb, ib, nb)
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), (step, k)
        a.upload(ha, na, True)
        b.upload(hb, nb, True)
    pa, pb = a.profile(False), b.profile(False)
    assert pa["n_speculative"] > 0 and pa["n_speculative"] == pb["n_speculative"]
    # every exchange after a speculative step that stood overlapped its solve
    assert pa["n_overlapped"] == 2 * (pa["n_speculative"] - pa["n_undone"]), pa
    assert pb["n_overlapped"] == 0, pb
    qa, qb = by_id(a.get_particles()), by_id(b.get_particles())
    for k in qa:
        assert np.array_equal(qa[k], qb[k]), k
