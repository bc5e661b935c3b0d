"""Pins of the oracle's fixed-point CIC deposit (Sec. 2.1.3) and the
fixed-point to space-charge conversion."""
import numpy as np
import pytest

import oracle as O
import workloads as W

S = 2.0 ** 32


@pytest.mark.parametrize("prec", [64, 32])
def test_charge_conservation_exact(prec):
    grid = W.grid_spec(9, 7, 8, 2e-5, origin=(1e-5, 0, -3e-5))
    p0 = W.random_particles(3000, grid, 11, w_range=(0.5, 2000.0))
    m = O.Model(W.zero_gas(), 1e-12, 1, prec, grid)
    q = O.deposit(m, O.Particles(3000, p0))
    if prec == 64:
        expect = sum(int(np.rint(w * S)) for w in p0["w"])
    else:
        expect = sum(int(np.rint(np.float32(w) * np.float32(S))) for w in p0["w"])
    assert int(q.sum()) == expect
    assert q.min() >= 0


@pytest.mark.parametrize("prec", [64, 32])
def test_cell_centre_fills_one_cell_and_translation(prec):
    dx = 2.0 ** -13          # a power of two: cell centres are exact in binary32 too
    grid = W.grid_spec(8, 8, 8, dx)
    p0 = dict(x=np.array([(3 + 0.5) * dx]), y=np.array([(4 + 0.5) * dx]), z=np.array([(2 + 0.5) * dx]),
              w=np.array([3.0]), id=np.array([0], np.uint64))
    m = O.Model(W.zero_gas(), 1e-12, 1, prec, grid)
    q = O.deposit(m, O.Particles(1, p0)).reshape(8, 8, 8)
    assert q[2, 4, 3] == int(3 * S) and q.sum() == int(3 * S)
    # a general position, then shifted by whole cells: the pattern shifts
    base = dict(x=np.array([2.3125 * dx]), y=np.array([3.703125 * dx]), z=np.array([2.515625 * dx]),
                w=np.array([7.25]), id=np.array([0], np.uint64))
    q1 = O.deposit(m, O.Particles(1, base)).reshape(8, 8, 8)
    sh = dict(base, x=base["x"] + 2 * dx, z=base["z"] + dx)
    q2 = O.deposit(m, O.Particles(1, sh)).reshape(8, 8, 8)
    assert np.array_equal(np.roll(np.roll(q1, 2, axis=2), 1, axis=0)[3:7, 2:6, 3:7], q2[3:7, 2:6, 3:7])
    # bilinear fractions: the corner weights equal the CIC products
    f = np.array([0.8125, 0.203125, 0.015625])
    cell = q1[2, 3, 1] / (7.25 * S)
    assert abs(cell - (1 - f[0]) * (1 - f[1]) * (1 - f[2])) < 1e-12


def test_wall_folding_conserves():
    grid = W.grid_spec(4, 4, 4, 1e-4)
    p0 = dict(x=np.array([0.1e-4]), y=np.array([3.95e-4]), z=np.array([0.0]), w=np.array([1.0]),
              id=np.array([0], np.uint64))
    m = O.Model(W.zero_gas(), 1e-12, 1, 64, grid)
    q = O.deposit(m, O.Particles(1, p0)).reshape(4, 4, 4)
    assert q.sum() == int(S)
    assert q[0, 3, 0] == int(S)   # half a cell from every wall it touches: all folds into the corner cell


def test_fixed_to_rho():
    dV = 8e-15
    qe = np.array([0, int(S), 3 * int(S)], np.int64)
    qp = np.array([int(S), int(S), int(S)], np.int64)
    qn = np.array([0, 0, int(S) // 2], np.int64)
    rho = O.fixed_to_rho(dV, qe, qp, qn)
    assert np.allclose(rho, O.Q_E / dV * np.array([1.0, 0.0, -2.5]), rtol=1e-15)


def test_binary32_corner_weights_against_float64():
    """The error the single-precision path's binary32 deposit (Sec. 2.1.3)
    makes against the float64 CIC, stated per particle: the cell coordinate
    (x - ox) / dx of a grid of n cells is formed in binary32 with an absolute
    error of at most ~1.5 n 2^-24, which each of a corner's three factors
    carries, so every corner weight lies within 3 (1.5 n 2^-24 + 2^-23) of the
    particle's weight (measured: at most 1.2e-5, median 2.3e-6 at n = 128);
    the charge is conserved exactly in both (the eighth corner takes the
    remainder) and totals agree for weights held in float32."""
    n = 128
    grid = W.grid_spec(n, n, n, 20e-6)
    p0 = W.random_particles(400, grid, 5, w_range=(1.0, 500.0))
    p = dict(p0)
    for k in ("x", "y", "z", "w"):
        p[k] = np.asarray(p0[k], np.float32).astype(np.float64)  # the state the float32 path holds
    m32 = O.Model(W.zero_gas(), 1e-12, 1, 32, grid)
    m64 = O.Model(W.zero_gas(), 1e-12, 1, 64, grid)
    bound = 3 * (1.5 * n * 2.0 ** -24 + 2.0 ** -23)
    worst = 0.0
    for i in range(len(p["x"])):
        pi = {k: np.asarray(v[i:i + 1]) for k, v in p.items()}
        a = O.deposit(m32, O.Particles(1, pi))
        b = O.deposit(m64, O.Particles(1, pi))
        assert int(a.sum()) == int(b.sum())
        worst = max(worst, float(np.abs(a - b).max()) / (pi["w"][0] * S))
    assert worst <= bound, (worst, bound)
    assert worst > 0.0   # the binary32 path is not the float64 one
