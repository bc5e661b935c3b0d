"""Pins of the oracle's mover (Eqs. 1-2, velocity Verlet) and field gather
(Sec. 2.1.3, trilinear interpolation) against closed forms."""
import numpy as np

import oracle as O
import workloads as W

QM = O.Q_E / O.M_ELEC


def test_ballistic_uniform_field_many_steps():
    """No collisions, constant a: x = x0 + v0 t + a t^2/2, v = v0 + a t exactly."""
    g = W.zero_gas()
    E0 = np.array([1e5, -2e5, 3e5])
    m = O.Model(g, 1e-12, 7, 64, None, None, E0=tuple(E0))
    p0 = W.random_particles(50, None, 1, box=([0, 0, 0], [1e-3] * 3))
    p = O.Particles(100, p0)
    n = 300
    for s in range(1, n + 1):
        rc, st = O.step(m, p, s, s == 1)
        assert rc == 0 and st.n_null == 0 and st.n_events == 0
    v = p.view()
    a = -QM * E0
    t = n * 1e-12
    for d, (xk, vk) in enumerate((("x", "vx"), ("y", "vy"), ("z", "vz"))):
        xe = p0[xk] + p0[vk] * t + 0.5 * a[d] * t * t
        ve = p0[vk] + a[d] * t
        assert np.allclose(v[xk], xe, rtol=1e-12, atol=1e-15)
        assert np.allclose(v[vk], ve, rtol=1e-12, atol=1e-6)
        assert np.allclose(v["a" + xk], a[d], rtol=1e-15)


def test_verlet_with_changing_field():
    """Eq. 2: after the correction at the start of step n+1,
    v = v(t) + dt/2 (a(t) + a(t+dt)); Eq. 1: x(t+dt) = x + dt v + dt^2 a(t)/2."""
    g = W.zero_gas()
    grid = W.grid_spec(4, 4, 4, 1e-3)
    dt = 1e-11
    E1 = (np.full((4, 4, 4), 2e5, np.float32), np.full((4, 4, 4), -1e5, np.float32),
          np.full((4, 4, 4), 5e4, np.float32))
    E2 = tuple((f * np.float32(-3.0)).astype(np.float32) for f in E1)
    p0 = W.random_particles(20, grid, 2, vmax=1e4, box=([1.5e-3] * 3, [2.5e-3] * 3))
    p = O.Particles(40, p0)
    m1 = O.Model(g, dt, 3, 64, grid, E1)
    m2 = O.Model(g, dt, 3, 64, grid, E2)
    O.step(m1, p, 1, True)
    O.step(m2, p, 2, False)
    v = p.view()
    a1 = -QM * np.array([float(f[0, 0, 0]) for f in E1])
    a2 = -QM * np.array([float(f[0, 0, 0]) for f in E2])
    for d, (xk, vk) in enumerate((("x", "vx"), ("y", "vy"), ("z", "vz"))):
        x1 = p0[xk] + dt * p0[vk] + 0.5 * dt * dt * a1[d]            # Eq. 1
        v1 = p0[vk] + 0.5 * dt * (a1[d] + a2[d])                     # Eq. 2
        x2 = x1 + dt * v1 + 0.5 * dt * dt * a2[d]
        v2 = v1 + dt * a2[d]
        assert np.allclose(v[xk], x2, rtol=1e-12, atol=1e-18)
        assert np.allclose(v[vk], v2, rtol=1e-12, atol=1e-9)


def test_gather_reproduces_linear_field_and_clamps():
    grid = W.grid_spec(6, 5, 7, 1e-4, origin=(1e-4, -2e-4, 3e-4))
    G = np.array([[1e8, -2e8, 3e8], [0.5e8, 1e8, -1e8], [2e8, 0.0, 1e8]])
    c0 = np.array([1e4, -3e4, 2e4])
    F = W.linear_field(grid, G, c0)
    m = O.Model(W.zero_gas(), 1e-12, 1, 64, grid, F)
    rng = np.random.default_rng(0)
    lo = np.array(grid["origin"]) + 0.5 * grid["dx"]
    hi = np.array(grid["origin"]) + (np.array([6, 5, 7]) - 0.5) * grid["dx"]
    X = lo + (hi - lo) * rng.random((200, 3))
    E = O.gather_field(m, X[:, 0], X[:, 1], X[:, 2])
    # exact value of the float32-rounded nodal field, interpolated: compare with the
    # linear field itself at the tolerance of the float32 node rounding
    Ee = c0 + X @ G.T
    assert np.allclose(E, Ee, rtol=2e-7, atol=2e-7 * np.abs(Ee).max())
    # outer half cell: constant extrapolation of the boundary layer
    Xo = np.array([[grid["origin"][0] + 0.1 * grid["dx"], lo[1], lo[2]]])
    Xi = np.array([[lo[0], lo[1], lo[2]]])
    assert np.array_equal(O.gather_field(m, *Xo.T), O.gather_field(m, *Xi.T))


def test_specular_reflection_at_faces():
    g = W.zero_gas()
    grid = W.grid_spec(4, 4, 4, 1e-4)
    L = 4e-4
    zero = tuple(np.zeros((4, 4, 4), np.float32) for _ in range(3))
    m = O.Model(g, 1e-11, 1, 64, grid, zero)
    p0 = dict(x=np.array([0.5e-4]), y=np.array([3.9e-4]), z=np.array([2e-4]),
              vx=np.array([-1e7]), vy=np.array([2e6]), vz=np.array([0.0]),
              w=np.array([1.0]), id=np.array([5], np.uint64))
    p = O.Particles(4, p0)
    O.step(m, p, 1, True)
    v = p.view()
    # x: 0.5e-4 - 1e-4 = -0.5e-4 -> reflected to 0.5e-4 with vx negated
    assert np.isclose(v["x"][0], 0.5e-4, rtol=1e-12) and v["vx"][0] == 1e7
    # y: 3.9e-4 + 0.2e-4 = 4.1e-4 -> 2L - y = 3.9e-4
    assert np.isclose(v["y"][0], 2 * L - 4.1e-4, rtol=1e-12) and v["vy"][0] == -2e6


def test_gather_of_a_float64_field_is_exact_for_a_linear_field():
    """The same gather from float64 nodes: a linear field is reproduced to
    rounding (no float32 node error left)."""
    grid = W.grid_spec(6, 5, 7, 1e-4, origin=(1e-4, -2e-4, 3e-4))
    G = np.array([[1e8, -2e8, 3e8], [0.5e8, 1e8, -1e8], [2e8, 0.0, 1e8]])
    c0 = np.array([1e4, -3e4, 2e4])
    z, y, x = np.meshgrid(*(grid["origin"][d] + (np.arange(n) + 0.5) * grid["dx"]
                            for d, n in ((2, 7), (1, 5), (0, 6))), indexing="ij")
    F = tuple(np.ascontiguousarray(c0[d] + G[d][0] * x + G[d][1] * y + G[d][2] * z) for d in range(3))
    m = O.Model(W.zero_gas(), 1e-12, 1, 64, grid, F)
    rng = np.random.default_rng(1)
    lo = np.array(grid["origin"]) + 0.5 * grid["dx"]
    hi = np.array(grid["origin"]) + (np.array([6, 5, 7]) - 0.5) * grid["dx"]
    X = lo + (hi - lo) * rng.random((200, 3))
    E = O.gather_field(m, X[:, 0], X[:, 1], X[:, 2])
    Ee = c0 + X @ G.T
    assert np.allclose(E, Ee, rtol=1e-13, atol=1e-13 * np.abs(Ee).max())


def test_verlet_half_kick_uses_the_previous_steps_length():
    """Eq. 2 over a step of length dt1 followed by one of dt2: the correction at
    the start of the second step is dt1/2 (a(t) + a(t + dt1)) - dt1 a(t), then
    the second flight adds dt2 a(t + dt1)."""
    g = W.zero_gas()
    grid = W.grid_spec(4, 4, 4, 1e-3)
    dt1, dt2 = 1e-11, 0.6e-11
    E1 = tuple(np.full((4, 4, 4), v, np.float32) for v in (2e5, -1e5, 5e4))
    E2 = tuple((f * np.float32(-3.0)).astype(np.float32) for f in E1)
    p0 = W.random_particles(20, grid, 2, vmax=1e4, box=([1.5e-3] * 3, [2.5e-3] * 3))
    p = O.Particles(40, p0)
    O.step(O.Model(g, dt1, 3, 64, grid, E1), p, 1, True)
    O.step(O.Model(g, dt2, 3, 64, grid, E2, dt_kick=dt1), p, 2, False)
    v = p.view()
    a1 = -QM * np.array([float(f[0, 0, 0]) for f in E1])
    a2 = -QM * np.array([float(f[0, 0, 0]) for f in E2])
    for d, (xk, vk) in enumerate((("x", "vx"), ("y", "vy"), ("z", "vz"))):
        x1 = p0[xk] + dt1 * p0[vk] + 0.5 * dt1 * dt1 * a1[d]
        v1 = p0[vk] + 0.5 * dt1 * (a1[d] + a2[d])
        x2 = x1 + dt2 * v1 + 0.5 * dt2 * dt2 * a2[d]
        v2 = v1 + dt2 * a2[d]
        assert np.allclose(v[xk], x2, rtol=1e-12, atol=1e-18)
        assert np.allclose(v[vk], v2, rtol=1e-12, atol=1e-9)
