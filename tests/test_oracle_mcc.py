"""Closed-form pins of the oracle's null-collision Monte Carlo (Sec. 2.1.1)
and of its swarm coefficients (Sec. 2.2.2).

Constant-frequency gases have exact moment equations: with lab-isotropic
scattering the post-collision mean velocity is zero, so
d<v>/dt = a - nu0 <v>  ->  <v_z>(t) = W (1 - exp(-nu0 t)) from rest, W = eE/(m nu0);
elastic loss (2 m/M)(1 - cos chi) with <cos chi> = 0 gives the steady energy
<eps> = M W^2 / 2; a constant ionization frequency gives E[N] = N0 exp(nu t)
(Yule process, variance N0 e^{nu t}(e^{nu t} - 1)); a constant attachment
frequency gives E[N] = N0 exp(-nu t) (binomial)."""
import numpy as np

import oracle as O
import workloads as W

QM = O.Q_E / O.M_ELEC


def _cold(n):
    z = np.zeros(n)
    return dict(x=z, y=z, z=z, vx=z, vy=z, vz=z, w=np.ones(n), id=np.arange(n, dtype=np.uint64))


def test_constant_nu_drift_relaxation():
    nu0, E = 1e12, 2e5
    gas = W.single_process_gas(W.ELASTIC, nu0 / W.N_GAS, mass=0.0)
    dt = 0.5e-12
    m = O.Model(gas, dt, 21, 64, None, None, E0=(0.0, 0.0, -E))
    assert abs(m.nu_max - nu0) / nu0 < 1e-12
    n = 40000
    p = O.Particles(n, _cold(n))
    Wd = QM * E / nu0
    for s in range(1, 9):
        rc, st = O.step(m, p, s, s == 1)
        assert st.n_null == 0
        vz = p.view()["vz"]
        t = s * dt
        expect = Wd * (1 - np.exp(-nu0 * t))
        err = vz.std() / np.sqrt(n)
        assert abs(vz.mean() - expect) < 4.5 * err, (s, vz.mean(), expect, err)
        # transverse drift vanishes
        vx = p.view()["vx"]
        assert abs(vx.mean()) < 4.5 * vx.std() / np.sqrt(n)


def test_energy_balance_finite_mass():
    nu0, M = 1e12, 100 * O.M_ELEC
    Wd = 1e5
    E = Wd * nu0 / QM
    gas = W.single_process_gas(W.ELASTIC, nu0 / W.N_GAS, mass=M)
    mom, cnt, res, m = O.swarm(gas, 0.0, 5000, 600, 1e-12, 33, E_override=E, kT_eV=0.5)
    eps_ss = M * Wd ** 2 / 2 / O.Q_E
    tail = mom[400:, 13] / mom[400:, 0]
    assert abs(tail.mean() - eps_ss) / eps_ss < 0.03
    assert abs(res[0] - Wd) / Wd < 0.03           # flux drift = eE/(m nu0)
    assert abs(res[1] - Wd) / Wd < 0.06           # bulk drift equals it without growth


def test_growth_constant_ionization():
    nu_i = 1e10
    gas = W.single_process_gas(W.IONIZATION, nu_i / W.N_GAS, threshold=0.0)
    n0, steps, dt = 4000, 100, 1e-12
    mom, cnt, res, m = O.swarm(gas, 0.0, n0, steps, dt, 44, n_lo=1, n_hi=10 ** 9, E_override=1e5)
    t = steps * dt
    g = np.exp(nu_i * t)
    sd = np.sqrt(n0 * g * (g - 1))
    assert abs(cnt[-1] - n0 * g) < 4 * sd
    # event weights per step integrate to the growth
    assert abs(mom[:, 14].sum() - (cnt[-1] - n0)) < 1e-9


def test_loss_constant_attachment():
    nu_a = 1e10
    gas = W.single_process_gas(W.ATTACHMENT, nu_a / W.N_GAS)
    n0, steps, dt = 10000, 100, 1e-12
    mom, cnt, res, m = O.swarm(gas, 0.0, n0, steps, dt, 45, n_lo=1, n_hi=10 ** 9, E_override=1e5)
    pr = np.exp(-nu_a * steps * dt)
    assert abs(cnt[-1] - n0 * pr) < 4 * np.sqrt(n0 * pr * (1 - pr))
    assert abs(mom[:, 15].sum() - (n0 - cnt[-1])) < 1e-9


def test_null_fraction_matches_rate_ratio():
    """Two constant processes with nu_1 + nu_2 = nu_max: no nulls; one process
    with half of nu_max at the top node only: the real-collision fraction of
    candidate events equals nu(eps)/nu_max."""
    nu0 = 1e12
    a = W.single_process_gas(W.ELASTIC, 0.3 * nu0 / W.N_GAS, mass=0.0)
    b = W.single_process_gas(W.EXCITATION, 0.7 * nu0 / W.N_GAS, threshold=0.0)
    gas = W.multi_gas([a, b])
    m = O.Model(gas, 1e-12, 9, 64, None, None, E0=(0, 0, -1e4))
    n = 5000
    p = O.Particles(n, _cold(n))
    tot = np.zeros(2)
    ev = 0
    for s in range(1, 6):
        rc, st = O.step(m, p, s, s == 1)
        tot += np.array(st.n_coll[:2])
        ev += st.n_events
        assert st.n_null == 0
    frac = tot[0] / tot.sum()
    assert abs(frac - 0.3) < 4 * np.sqrt(0.21 / tot.sum())


def test_flux_equals_bulk_for_constant_ionization():
    nu0, nu_i, M = 1e12, 2e10, 100 * O.M_ELEC
    gas = W.multi_gas([W.single_process_gas(W.ELASTIC, nu0 / W.N_GAS, mass=M),
                       W.single_process_gas(W.IONIZATION, nu_i / W.N_GAS, threshold=0.0)])
    E = 1e5 * nu0 / QM
    mom, cnt, res, m = O.swarm(gas, 0.0, 3000, 400, 1e-12, 46, n_lo=1000, n_hi=6000, E_override=E)
    sig = np.hypot(res[11], res[12])
    assert abs(res[1] - res[0]) < 4 * sig + 0.01 * res[0]


def test_bulk_exceeds_flux_in_ionizing_air():
    """The paper reports bulk mobility above flux mobility in high fields where
    ionization dominates (Sec. 2.2.2); the synthetic air shows the same at 300 Td."""
    gas = W.synthetic_air()
    mom, cnt, res, m = O.swarm(gas, 300.0, 2000, 400, 1e-12, 5, n_lo=1000, n_hi=4000)
    assert res[1] - res[0] > 4 * np.hypot(res[11], res[12])
    assert res[9] > 0 and res[7] > 0
