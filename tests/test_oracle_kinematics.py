"""Pins of the oracle's collision kinematics (Sec. 2.1.1) and of its swarm
coefficients and resampling (Sec. 2.2.2) by exact properties.

Forced collisions: a one-process gas with a constant rate nu (so nu_max = nu
and every candidate event is real) and no field (speeds change only at
collisions).
- Excitation removes the threshold energy: every final energy is
  eps0 - k eps_th for a whole k, and the k add up to the collision count.
- Ionization shares the remaining energy equally: a primary of energy e
  leaves two electrons of (e - eps_ion)/2 each, so the final energies lie on
  the ladder e_{L+1} = (e_L - eps_ion)/2 and the numbers N_L of electrons on
  each rung satisfy sum_L N_L 2^-L = N0 (each event replaces a leaf of a
  binary tree by two leaves one level down).

Finite-mass elastic swarm with a constant nu (closed forms from the moment
equations of the elastic rule eps' = eps (1 - 2 r (1 - cos chi)), r = m/M,
with the new direction isotropic): a collision keeps the fraction
f(r) = <c sqrt(1 - 2r(1 - c))> (c = cos chi uniform on [-1, 1]) of the
velocity, so momentum relaxes at nu_m = nu (1 - f); it keeps the fraction
1 - 2r of <v^2>, and of <v_x^2> the value (1 - 2r) <v^2> / 3.  In the steady
state, with a = eE/m:
  W = a / nu_m,  <v^2> = a W / (r nu),
  D_T = (1 - 2r) <v^2> / (3 nu_m),
  D_L = (2 a W / nu + (1 - 2r) <v^2> / 3 - W^2) / nu_m,
and without growth or loss the bulk coefficients equal the flux ones.

Resampling: thinning keeps each electron with probability 1/2 and
duplication copies every electron, neither changing weights, so counts halve
(binomially) or double (exactly) and the rate coefficients stay unbiased.
The rate coefficients divide each step's event weight by the time integral
of the swarm weight over that step; with nu dt = 0.1-0.2 here, dividing by
the end-of-step weight instead would be off by 5-10 %."""
import numpy as np
from scipy import integrate

import oracle as O
import workloads as W

QM = O.Q_E / O.M_ELEC


def _mono(n, eps_eV, seed):
    """n electrons at the origin with energy eps_eV in isotropic directions."""
    r = np.random.default_rng(seed)
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    sp = np.sqrt(2 * O.Q_E * eps_eV / O.M_ELEC)
    z = np.zeros(n)
    return dict(x=z, y=z, z=z, vx=sp * d[:, 0], vy=sp * d[:, 1], vz=sp * d[:, 2], w=np.ones(n),
                id=np.arange(n, dtype=np.uint64))


def _energies(p):
    v = p.view()
    return 0.5 * O.M_ELEC * (v["vx"] ** 2 + v["vy"] ** 2 + v["vz"] ** 2) / O.Q_E


def test_forced_excitation_removes_the_threshold():
    nu, dt, th, e0, n = 3e12, 1e-12, 6.2, 100.0, 4000
    gas = W.single_process_gas(W.EXCITATION, nu / W.N_GAS, threshold=th)
    m = O.Model(gas, dt, 71, 64, None, None, E0=(0.0, 0.0, 0.0))
    assert abs(m.nu_max - nu) / nu < 1e-12
    p = O.Particles(n, _mono(n, e0, 1))
    rc, st = O.step(m, p, 1, True)
    assert rc == 0 and st.n_null == 0 and st.n_coll[0] > 2 * n
    e = _energies(p)
    k = np.rint((e0 - e) / th)
    assert np.all(k >= 0) and k.max() <= e0 / th
    assert np.allclose(e, e0 - k * th, rtol=0, atol=1e-9 * e0)
    assert int(k.sum()) == st.n_coll[0]
    # the new directions are isotropic: no memory of the initial ones
    v = p.view()
    sp = np.sqrt(v["vx"] ** 2 + v["vy"] ** 2 + v["vz"] ** 2)
    for c in ("vx", "vy", "vz"):
        assert abs(np.mean(v[c] / sp)) < 4 * np.sqrt(1 / 3 / n)


def test_forced_ionization_shares_the_remaining_energy_equally():
    nu, dt, th, e0, n = 4e11, 1e-12, 15.6, 200.0, 20000
    gas = W.single_process_gas(W.IONIZATION, nu / W.N_GAS, threshold=th)
    m = O.Model(gas, dt, 72, 64, None, None, E0=(0.0, 0.0, 0.0))
    p = O.Particles(8 * n, _mono(n, e0, 2))
    rc, st = O.step(m, p, 1, True)
    assert rc == 0 and st.n_null == 0
    ladder = [e0]
    while ladder[-1] > th:
        ladder.append((ladder[-1] - th) / 2)
    # 200 -> 92.2 -> 38.3 -> 11.35; an event below the threshold leaves two electrons at rest
    # (depth 4 or more), which is rare at nu dt = 0.4
    e = _energies(p)
    lvl = np.full(len(e), -1)
    for L, eL in enumerate(ladder):
        lvl[np.abs(e - eL) <= 1e-9 * e0] = L
    zero = e == 0.0
    assert np.all((lvl >= 0) | zero), np.unique(e[(lvl < 0) & ~zero])[:5]
    NL = np.bincount(lvl[lvl >= 0], minlength=len(ladder))
    assert len(ladder) == 4 and NL[1] > 1000 and NL[2] > 100 and zero.sum() < 0.05 * n
    rest = n - np.sum(NL * 2.0 ** -np.arange(len(NL)))
    assert 0.0 <= rest <= zero.sum() / 16 and (rest == 0.0) == (zero.sum() == 0)
    assert p.n == n + st.n_children and st.n_children == st.n_coll[0]


def test_finite_mass_swarm_matches_the_moment_closed_forms():
    nu, M, Wd0 = 1e12, 20 * O.M_ELEC, 1e5
    r = O.M_ELEC / M
    a = Wd0 * nu
    E = a / QM
    f = integrate.quad(lambda c: 0.5 * c * np.sqrt(1 - 2 * r * (1 - c)), -1, 1, epsabs=1e-14)[0]
    nu_m = nu * (1 - f)
    Wd = a / nu_m
    v2 = a * Wd / (r * nu)
    DT = (1 - 2 * r) * v2 / (3 * nu_m)
    DL = (2 * a * Wd / nu + (1 - 2 * r) * v2 / 3 - Wd ** 2) / nu_m
    eps = 0.5 * O.M_ELEC * v2 / O.Q_E
    gas = W.single_process_gas(W.ELASTIC, nu / W.N_GAS, mass=M)
    mom, cnt, res, m = O.swarm(gas, 0.0, 10000, 2000, 1e-12, 73, E_override=E, kT_eV=eps / 1.5)
    # (value, closed form, one-sigma error index); the bulk spreads are the least precise
    for name, i, ref in (("W_flux", 0, Wd), ("W_bulk", 1, Wd), ("DL_flux", 2, DL), ("DT_flux", 3, DT),
                         ("DL_bulk", 4, DL), ("DT_bulk", 5, DT), ("mean_eps", 6, eps)):
        sig = res[11 + i]
        assert abs(res[i] - ref) <= 4 * sig + 1e-3 * abs(ref), (name, res[i], ref, sig)
    # precise enough to tell the finite-mass corrections apart: f moves W by 1.8 % (and the bounds
    # hold it to 0.3 %), 1 - 2r moves D_L and D_T by 10 % (held to 3 %)
    assert res[11] < 0.003 * Wd and res[14] < 0.03 * DT and res[13] < 0.03 * DL


def test_thinning_halves_counts_and_keeps_the_ionization_rate():
    nu_i, dt, n0, n_hi = 2e11, 1e-12, 2000, 3000
    gas = W.multi_gas([W.single_process_gas(W.ELASTIC, 1e12 / W.N_GAS, mass=0.0),
                       W.single_process_gas(W.IONIZATION, nu_i / W.N_GAS, threshold=0.0)])
    mom, cnt, res, m = O.swarm(gas, 0.0, n0, 400, dt, 74, n_lo=10, n_hi=n_hi, E_override=1e5)
    thin = np.nonzero(cnt[:-1] > n_hi)[0]
    assert len(thin) >= 10
    g = np.exp(nu_i * dt)
    before, after = cnt[thin].astype(float), cnt[thin + 1].astype(float)
    # after = Binomial(before, 1/2) grown for one step (Yule: variance N g (g - 1))
    expect = (before / 2 * g).sum()
    var = (before / 4 * g ** 2 + before / 2 * g * (g - 1)).sum()
    assert abs(after.sum() - expect) < 4 * np.sqrt(var)
    # weights are not touched: the swarm weight is the count
    assert np.all(mom[:, 0] == cnt)
    k_exp = nu_i / W.N_GAS
    assert abs(res[7] - k_exp) <= 4 * res[18] + 1e-3 * k_exp, (res[7], k_exp, res[18])


def test_duplication_doubles_counts_and_keeps_the_attachment_rate():
    nu_a, dt, n0, n_lo = 1e11, 1e-12, 1000, 800
    gas = W.multi_gas([W.single_process_gas(W.ELASTIC, 1e12 / W.N_GAS, mass=0.0),
                       W.single_process_gas(W.ATTACHMENT, nu_a / W.N_GAS)])
    mom, cnt, res, m = O.swarm(gas, 0.0, n0, 400, dt, 75, n_lo=n_lo, n_hi=10 ** 9, E_override=1e5)
    dup = np.nonzero(cnt[:-1] < n_lo)[0]
    assert len(dup) >= 5
    # duplication is exact: the next step starts from 2N electrons and loses its attached weight
    assert np.all(cnt[dup + 1] == 2 * cnt[dup] - np.rint(mom[dup + 1, 15]).astype(np.int64))
    assert np.all(mom[:, 0] == cnt)
    k_exp = nu_a / W.N_GAS
    assert abs(res[8] - k_exp) <= 4 * res[19] + 1e-3 * k_exp, (res[8], k_exp, res[19])
