"""Pins of the oracle against values the paper prints (tests/golden/
paper_printed_values.txt): the E/N unit of Sec. 2.3, observed through the
oracle's swarm as the acceleration of collisionless electrons, and the
photon yield of Eq. 6 with the constants of Sec. 2.4, observed through the
oracle's emission draws."""
import os

import numpy as np

import oracle as O
import workloads as W

K_B = 1.380649e-23   # J/K (SI, exact)
Q_E, M_E = 1.602176634e-19, 9.1093837015e-31


def _golden():
    vals = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, rest = line.split("=", 1)
        value, section, digits = (f.strip() for f in rest.split(";"))
        vals[name.strip()] = (float(value), section, digits)
    return vals


def _half_unit(value, digits):
    """Half a unit in the last printed digit (relative), 0 for exact values."""
    if digits == "exact":
        return 0.0
    e = np.floor(np.log10(abs(value)))
    return 0.5 * 10.0 ** (e - int(digits) + 1) / abs(value)


def test_gas_density_is_the_ideal_gas_value():
    g = _golden()
    n, _, dig = g["n_gas_m3"]
    p = g["pressure_bar"][0] * 1e5
    T = g["temperature_K"][0]
    assert abs(p / (K_B * T) - n) / n <= _half_unit(n, dig)
    assert W.N_GAS_PAPER == n


def test_td_unit_through_the_oracle_swarm():
    """Collisionless electrons at E/N = 4.14 Td and the paper's density gain
    e E / m_e of speed per second along the field: E must be 1 kV/cm within
    the rounding of the two printed numbers (a wrong Td factor, density or
    field sign fails this)."""
    g = _golden()
    n, _, dn = g["n_gas_m3"]
    td, _, dtd = g["td_per_kV_cm"]
    gas = W.single_process_gas(W.ELASTIC, 0.0, n_gas=n)
    dt = 1e-12
    mom, _, _, _ = O.swarm(gas, td, 200, 6, dt, 7, n_lo=10, n_hi=10 ** 6)
    vz = mom[:, 9] / mom[:, 0]                       # weighted mean v_z per step
    accel = np.diff(vz) / dt
    assert np.allclose(accel, accel[0], rtol=1e-9)   # exact constant-field flights
    E = accel[0] * M_E / Q_E                         # electrons move against E = -E_z z
    assert E > 0
    tol = _half_unit(td, dtd) + _half_unit(n, dn) + 1e-9
    assert abs(E - 1e5) / 1e5 <= tol, (E, tol)


def test_photon_yield_of_eq6():
    """Eq. 6 with xi = 0.075 and p_q = 40 mbar at 1 bar: each ionization emits
    a photon with probability xi p_q / (p + p_q) = 0.002885.  1.6e7 emission
    draws of the oracle agree within 4 standard deviations (0.47 % each), which
    separates it from xi p_q / p (4 % higher) and from xi alone."""
    g = _golden()
    xi = g["xi"][0]
    pq = g["p_q_mbar"][0] * 100.0
    p = g["pressure_bar"][0] * 1e5
    gas = W.single_process_gas(W.IONIZATION, 1e-15, n_gas=W.N_GAS_PAPER)
    m = O.Model(gas, 1e-12, 2110144940, photo=dict(xi=xi, pq=pq, pressure=p, p_o2=0.2 * p,
                                                  chi_min=1.0, chi_max=2.0))
    emitted = n = 0
    for pid in range(1, 17):
        em, _, _ = O.photon_draws(m, pid, 3, 1_000_000)
        emitted += int(em.sum())
        n += em.size
    prob = xi * pq / (p + pq)
    sigma = np.sqrt(prob * (1 - prob) / n)
    assert abs(emitted / n - prob) <= 4 * sigma, (emitted / n, prob, sigma)
    assert abs(emitted / n - xi * pq / p) > 4 * sigma
