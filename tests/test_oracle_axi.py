"""Pins of the oracle's axisymmetric Poisson solve (the paper's axisymmetric
geometry) against values fixed by mathematics: the linear potential between
plates, Gauss's law through the physical ring-face areas, and second-order
convergence to a Bessel-sine solution."""
import numpy as np
import pytest

import oracle as O

special = pytest.importorskip("scipy.special")


def test_plates_only_linear():
    nr, nz, h, V = 12, 40, 1e-4, 700.0
    phi, rr, it = O.poisson_axi(nr, nz, h, np.zeros(nr * nz), None, 0.0, 0.0, V)
    z = (np.arange(nz) + 0.5) / nz
    assert np.abs(phi - V * z[:, None]).max() < 1e-9 * V


def test_gauss_law_through_ring_faces():
    """The flux of grad(phi) out of the z plates (ring areas pi (2i + 1) h^2,
    half-cell gradients) equals -Q / eps0 with Q = sum rho pi (2i + 1) h^3;
    the outer cylinder carries none.  Holds for the discrete solution only if
    the operator is the conservative ring-cell form."""
    nr, nz, h = 16, 24, 5e-5
    r = np.random.default_rng(2)
    rho = r.normal(0, 1e-2, (nz, nr))
    phi, rr, it = O.poisson_axi(nr, nz, h, rho, None, 0.0, 0.0, 0.0)
    area = np.pi * (2 * np.arange(nr) + 1) * h * h
    flux = np.sum(area * (0.0 - phi[0]) / (h / 2)) + np.sum(area * (0.0 - phi[-1]) / (h / 2))
    Q = np.sum(rho * area[None, :] * h)
    assert abs(flux + Q / O.EPS_0) <= 1e-9 * abs(Q / O.EPS_0) + 1e-12


def test_second_order_convergence_to_bessel_solution():
    """phi* = J0(j1 r / R) sin(pi z / L) has no flux through r = R (J0' = -J1,
    j1 the first zero of J1), vanishes on the plates and satisfies -lap phi* =
    ((j1/R)^2 + (pi/L)^2) phi*.  The discrete error falls by ~4 per halving."""
    R, L = 1e-3, 2e-3
    j1 = special.jn_zeros(1, 1)[0]
    lam = (j1 / R) ** 2 + (np.pi / L) ** 2
    errs = []
    for nr in (8, 16, 32):
        nz = 2 * nr
        h = R / nr
        rc = (np.arange(nr) + 0.5) * h
        zc = (np.arange(nz) + 0.5) * h
        ex = special.j0(j1 * rc / R)[None, :] * np.sin(np.pi * zc / L)[:, None]
        phi, rr, it = O.poisson_axi(nr, nz, h, O.EPS_0 * lam * ex, None, 0.0, 0.0, 0.0)
        errs.append(np.abs(phi - ex).max())
    for a, b in zip(errs[:-1], errs[1:]):
        assert 3.0 < a / b < 5.0, errs
    assert errs[-1] < 2e-3
