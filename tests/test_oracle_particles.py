"""Pins of the oracle's initial seeding (Sec. 2.3, Eq. 7) and super-particle
weight update (Sec. 2.1.2, Eq. 3)."""
import numpy as np

import oracle as O
import workloads as W

S24 = 2.0 ** 24


def test_gaussian_seed_statistics():
    grid = W.grid_spec(24, 24, 24, 2e-5)
    L = 24 * 2e-5
    c = (0.5 * L, 0.5 * L, 0.4 * L)
    n0, R, w0 = 1e19, 1e-4, 100.0
    m = O.Model(W.zero_gas(), 1e-12, 77, 64, grid)
    p = O.seed_gaussian(m, n0, R, c, w0, 2_000_000)
    v = p.view()
    Z, Y, X = np.meshgrid(*((np.arange(24) + 0.5) * 2e-5,) * 3, indexing="ij")
    lam = n0 * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / R ** 2) * (2e-5) ** 3 / w0
    frac = lam - np.floor(lam)
    assert abs(p.n - lam.sum()) < 5 * np.sqrt((frac * (1 - frac)).sum()) + 1
    # integral of the Gaussian: n0 pi^{3/2} R^3 (the box holds nearly all of it)
    assert abs(p.n * w0 - n0 * np.pi ** 1.5 * R ** 3) / (n0 * np.pi ** 1.5 * R ** 3) < 0.02
    assert np.array_equal(v["id"], np.arange(p.n, dtype=np.uint64))
    assert np.all(v["vx"] == 0) and np.all(v["w"] == w0)
    # per-cell counts are floor(lambda) or floor(lambda) + 1
    ix = np.floor(v["x"] / 2e-5).astype(int)
    iy = np.floor(v["y"] / 2e-5).astype(int)
    iz = np.floor(v["z"] / 2e-5).astype(int)
    cnt = np.zeros((24, 24, 24), int)
    np.add.at(cnt, (iz, iy, ix), 1)
    d = cnt - np.floor(lam)
    assert d.min() >= 0 and d.max() <= 1


def test_seed_skips_mask():
    grid = W.grid_spec(16, 16, 16, 2e-5)
    L = 16 * 2e-5
    mask = W.needle_mask(grid, 0.1e-3, 0.06e-3)
    m = O.Model(W.zero_gas(), 1e-12, 1, 64, grid, mask=mask)
    p = O.seed_gaussian(m, 1e18, 1e-4, (0.5 * L, 0.5 * L, L - 0.1e-3), 20.0, 2_000_000)
    v = p.view()
    c = (np.floor(v["z"] / 2e-5).astype(int) * 16 + np.floor(v["y"] / 2e-5).astype(int)) * 16 + \
        np.floor(v["x"] / 2e-5).astype(int)
    assert not mask.ravel()[c].any()


def _cellw(v, grid):
    dx = grid["dx"]
    c = (np.floor(v["z"] / dx).astype(int) * grid["ny"] + np.floor(v["y"] / dx).astype(int)) * grid["nx"] + \
        np.floor(v["x"] / dx).astype(int)
    return c


def test_merge_split_invariants():
    grid = W.grid_spec(6, 6, 6, 1e-4)
    rng = np.random.default_rng(3)
    n = 6000
    p0 = W.random_particles(n, grid, 31, w_range=(1.0, 2.0))
    # a few heavy particles to split
    p0["w"][:40] = rng.uniform(200, 900, 40)
    m = O.Model(W.zero_gas(), 1e-12, 123, 64, grid)
    p = O.Particles(4 * n, p0)
    W0 = p0["w"].sum()
    rc, ms = O.merge_split(m, p, 9, n_ppc=10, w_min=1.0)
    assert rc == 0
    v = p.view()
    assert abs(v["w"].sum() - W0) / W0 < 1e-13
    assert len(np.unique(v["id"])) == p.n
    c = _cellw(v, grid)
    c0 = _cellw(p0, grid)
    for cell in np.unique(c0):
        Wc = np.rint(p0["w"][c0 == cell] * S24).sum() / S24
        om = max(Wc / 10, 1.0)
        ws = v["w"][c == cell]
        assert ws.max() <= 1.5 * om + 1e-12
        assert (ws < 2 * om / 3).sum() <= 1
        Wt = p0["w"][c0 == cell].sum()
        assert abs(ws.sum() - Wt) / Wt < 1e-12


def test_merge_keeps_state_of_a_member_and_split_copies_identical():
    grid = W.grid_spec(2, 2, 2, 1e-4)
    p0 = W.random_particles(200, grid, 12, w_range=(1.0, 1.5))
    p0["w"][0] = 1000.0
    m = O.Model(W.zero_gas(), 1e-12, 5, 64, grid)
    p = O.Particles(2000, p0)
    rc, ms = O.merge_split(m, p, 3, n_ppc=75, w_min=1.0)
    v = p.view()
    orig = {int(i): k for k, i in enumerate(p0["id"])}
    for k in range(p.n):
        i = int(v["id"][k])
        if i in orig:
            j = orig[i]
            assert v["x"][k] == p0["x"][j] and v["vz"][k] == p0["vz"][j]
    heavy = v["x"] == p0["x"][0]
    assert heavy.sum() > 1 and np.all(v["vx"][heavy] == p0["vx"][0])
    assert abs(v["w"][heavy].sum() - 1000.0) < 1e-12


def test_particle_cap_scales_omega():
    grid = W.grid_spec(4, 4, 4, 1e-4)
    p0 = W.random_particles(8000, grid, 13, w_range=(1.0, 1.0001))
    m = O.Model(W.zero_gas(), 1e-12, 5, 64, grid)
    p = O.Particles(20000, p0)
    rc, ms = O.merge_split(m, p, 3, n_ppc=75, w_min=1.0, cap=1000)
    assert ms.scale > 1
    assert p.n <= 1000 * 1.2 + 64
