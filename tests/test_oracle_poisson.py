"""Pins of the oracle's Poisson solve (Sec. 2.5: -lap(phi) = rho/eps0 on the
cell-centred grid, Dirichlet plates in z, Neumann elsewhere, electrode held at
its potential) and of E = -grad(phi)."""
import numpy as np

import oracle as O
import workloads as W


def _centres(grid):
    nx, ny, nz, h = grid["nx"], grid["ny"], grid["nz"], grid["dx"]
    return np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                       indexing="ij")


def test_manufactured_discrete_eigenfunction():
    """phi* = cos(pi x/Lx) cos(pi y/Ly) sin(pi z/Lz) satisfies the discrete
    Neumann (x, y) and homogeneous Dirichlet (z) ghost rules exactly and is an
    eigenvector of the 7-point Laplacian with eigenvalue
    lambda_h = sum_d (4/h^2) sin^2(pi h / (2 L_d)); so rho = eps0 lambda_h phi*
    has phi* as its exact discrete solution."""
    grid = W.grid_spec(12, 10, 14, 1e-4)
    h = grid["dx"]
    L = [grid["nx"] * h, grid["ny"] * h, grid["nz"] * h]
    Z, Y, X = _centres(grid)
    ph = np.cos(np.pi * X / L[0]) * np.cos(np.pi * Y / L[1]) * np.sin(np.pi * Z / L[2])
    lam = sum(4 / h ** 2 * np.sin(np.pi * h / (2 * Ld)) ** 2 for Ld in L)
    phi, rr, it = O.poisson(grid, O.EPS_0 * lam * ph, None, 0.0, 0.0, 0.0, rtol=1e-13)
    assert rr <= 1e-13
    assert np.abs(phi - ph).max() < 1e-10


def test_second_order_convergence_continuous_source():
    errs = []
    for n in (8, 16, 32):
        grid = W.grid_spec(n, n, n, 1.0 / n)
        Z, Y, X = _centres(grid)
        ex = np.cos(np.pi * X) * np.cos(2 * np.pi * Y) * np.sin(np.pi * Z)
        rho = O.EPS_0 * (np.pi ** 2 * (1 + 4 + 1)) * ex
        phi, rr, it = O.poisson(grid, rho, None, 0.0, 0.0, 0.0, rtol=1e-12)
        errs.append(np.abs(phi - ex).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3


def test_plates_only_linear_potential():
    grid = W.grid_spec(6, 5, 16, 1e-4)
    V0 = 5120.0
    phi, rr, it = O.poisson(grid, np.zeros((16, 5, 6)), None, 0.0, 0.0, V0, rtol=1e-14)
    L = 16 * 1e-4
    z = (np.arange(16) + 0.5) * 1e-4
    assert np.allclose(phi, (V0 * z / L)[:, None, None], rtol=0, atol=1e-9 * V0)
    Ex, Ey, Ez = O.grad_phi(grid, phi, 0.0, V0)
    assert np.allclose(Ez, -V0 / L, rtol=1e-9) and np.abs(Ex).max() < 1e-6 and np.abs(Ey).max() < 1e-6


def test_needle_mask_properties():
    grid = W.grid_spec(16, 16, 24, 1e-4)
    L = 24 * 1e-4
    V0 = 1000.0
    mask = W.needle_mask(grid, 0.8e-3, 0.25e-3)
    assert mask.sum() > 0
    phi, rr, it = O.poisson(grid, np.zeros((24, 16, 16)), mask, V0, 0.0, V0, rtol=1e-12)
    assert rr <= 1e-12
    assert np.all(phi[mask.astype(bool)] == V0)
    # maximum principle and the mirror symmetries of the geometry
    assert phi.min() >= -1e-9 and phi.max() <= V0 + 1e-9
    assert np.allclose(phi, phi[:, :, ::-1], atol=1e-8) and np.allclose(phi, phi[:, ::-1, :], atol=1e-8)
    # the needle raises the potential below its tip above the plate-only value
    k_tip = int(np.argmax(mask[:, 8, 8])) - 1
    z_tip = (k_tip + 0.5) * 1e-4
    assert phi[k_tip, 8, 8] > V0 * z_tip / L
