"""Pins of the oracle's photoionization (Sec. 2.4, discrete Monte Carlo
photons) against values fixed by mathematics: Zheleznyak's absorption
distribution through SciPy's exponential integral, the emission probability,
isotropy, and charge neutrality of every photoionization."""
import numpy as np
import pytest

import oracle as O
import workloads as W

special = pytest.importorskip("scipy.special")

TORR = 101325.0 / 760.0
CHI_MIN, CHI_MAX = 0.035 / (1e-3 * TORR), 2.0 / (1e-3 * TORR)   # 1/(m Pa)
P = 101325.0
P_O2 = 0.2 * P


def _model(prob, grid=None, mask=None, gas=None, field=None, boundary=0):
    pq = 4000.0
    xi = prob * (P + pq) / pq
    photo = dict(xi=xi, pq=pq, pressure=P, p_o2=P_O2, chi_min=CHI_MIN, chi_max=CHI_MAX)
    return O.Model(gas or W.synthetic_air(), 1e-12, 2110144940, 64, grid, field, mask=mask, boundary=boundary,
                   photo=photo)


def test_absorption_distance_follows_zheleznyak():
    """Kolmogorov-Smirnov against F(r) = 1 - (E1(a r) - E1(b r)) / ln(b/a), the
    integral of f(r) = (e^-ar - e^-br) / (r ln(b/a)); and the mean
    (1/a - 1/b) / ln(b/a)."""
    m = _model(1.0)
    n = 200_000
    em, r, _ = O.photon_draws(m, 12345, 7, n)
    assert em.all()
    a, b = CHI_MIN * P_O2, CHI_MAX * P_O2
    rs = np.sort(r)
    F = 1.0 - (special.exp1(a * rs) - special.exp1(b * rs)) / np.log(b / a)
    ks = np.max(np.maximum(np.arange(1, n + 1) / n - F, F - np.arange(n) / n))
    assert ks < 1.63 / np.sqrt(n), ks     # 1 % level
    mean = (1 / a - 1 / b) / np.log(b / a)
    # the distribution has a heavy tail (sd ~ 3x the mean): 5 standard errors
    sd = np.sqrt((1 / a ** 2 - 1 / b ** 2) / np.log(b / a) - mean ** 2)
    assert abs(r.mean() - mean) < 5 * sd / np.sqrt(n), (r.mean(), mean)


def test_emission_probability_and_isotropy():
    m = _model(0.3)
    n = 100_000
    em, r, d = O.photon_draws(m, 777, 3, n)
    k = em.sum()
    assert abs(k - 0.3 * n) < 4 * np.sqrt(n * 0.3 * 0.7)
    dirs = d[em]
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(dirs.mean(axis=0)) < 4 / np.sqrt(3 * k))
    assert np.all(np.abs((dirs ** 2).mean(axis=0) - 1 / 3) < 4 * np.sqrt(4 / 45 / k))
    assert np.all(r[~em] == 0.0)


def test_photoionization_is_charge_neutral():
    """Constant ionization frequency, reflecting faces, no electrode: every
    ionization and every absorbed photon creates one electron-ion pair, so
    the electron deposit minus the ion deposit is the initial charge
    exactly, and photoelectrons appear."""
    g = W.grid_spec(16, 16, 16, 1e-4)
    gas = W.single_process_gas(O.IONIZATION, 2e-14, threshold=0.0)
    m = _model(1.0, grid=g, gas=gas)
    p0 = W.random_particles(2000, g, 31, vmax=1e6, w_range=(1.0, 1.0))
    p = O.Particles(200000, p0)
    n = 16 ** 3
    qe, qp, qn = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64)
    rc, st = O.step(m, p, 1, True, qe, qp, qn)
    assert rc == 0
    assert st.n_children > 100 and st.n_photo > 0.5 * st.n_children
    assert int(qe.sum()) - int(qp.sum()) == 2000 * (1 << 32)
    assert p.n == 2000 + st.n_children + st.n_photo
