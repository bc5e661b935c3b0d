"""Pins of the oracle's rate table (Sec. 2.1.1 and 2.1.5: collision rates from
cross sections) and of its interpolation."""
import numpy as np

import oracle as O
import workloads as W


def test_speed_at_one_eV():
    """A single constant cross section sigma0 gives nu = N sigma0 v(eps); the
    electron speed at 1 eV is the textbook 5.931e5 m/s."""
    g = W.single_process_gas(W.ELASTIC, 0.0, n_bins=11, eps_min=0.01, eps_max=100.0)
    g["sigma"][:] = 1e-20
    nu, numax = O.rate_table(g)
    j = 5  # eps = 1 eV exactly on the log grid 0.01..100 with 11 nodes
    assert abs(g["eps"][j] - 1.0) < 1e-12
    v1 = nu[0, j] / (g["density"][0] * 1e-20)
    assert abs(v1 - 5.931e5) / 5.931e5 < 2e-4
    # nu grows as sqrt(eps): ratio between nodes 10 decades apart in eps
    assert np.allclose(nu[0, 1:] / nu[0, :-1], np.sqrt(g["eps"][1:] / g["eps"][:-1]), rtol=1e-12)
    assert numax == nu[0, -1]


def test_constant_rate_gas():
    g = W.single_process_gas(W.IONIZATION, 4e-16, n_bins=50)
    nu, numax = O.rate_table(g)
    assert np.allclose(nu, 4e-16 * W.N_GAS, rtol=1e-12)
    assert abs(numax - 4e-16 * W.N_GAS) / numax < 1e-12


def test_synthetic_air_thresholds_and_sum():
    g = W.synthetic_air()
    nu, numax = O.rate_table(g)
    for k in range(7):
        thr = g["threshold"][k]
        if thr > 0:
            assert np.all(nu[k, g["eps"] <= thr] == 0.0)
            assert np.any(nu[k] > 0)
    assert numax == np.max(nu.sum(axis=0))
    # the elastic rate tends to a constant at high energy: N sigma v ~ eps^-1/2 eps^1/2
    tail = nu[0, -50:]
    assert tail.max() / tail.min() < 1.02


def test_interpolation_linear_in_log_energy():
    g = W.synthetic_air(n_bins=101)
    m = O.Model(g, 1e-12, 1)
    eps = g["eps"]
    # nodes reproduce the table
    r = O.rates_at(m, eps[5:95])
    assert np.allclose(r.T, m.nu[:, 5:95], rtol=1e-9, atol=1e-12 * m.nu_max)
    # geometric midpoint of two nodes -> arithmetic mean of the node rates
    mid = np.sqrt(eps[10:90] * eps[11:91])
    r = O.rates_at(m, mid)
    assert np.allclose(r.T, 0.5 * (m.nu[:, 10:90] + m.nu[:, 11:91]), rtol=1e-9, atol=1e-6)
    # clamping below and above the table
    r = O.rates_at(m, np.array([0.0, 1e-5, 1e5]))
    assert np.array_equal(r[0], m.nu[:, 0]) and np.array_equal(r[1], m.nu[:, 0])
    assert np.array_equal(r[2], m.nu[:, -1])
