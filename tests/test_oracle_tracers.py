"""Pins for the oracle's dense velocity field (Eq. 3) and the tracer points
it carries along the shooting: the particle equations (the field at a
particle is its own velocity), closed forms, a high-order integrator of the
coupled system, linearity and symmetry."""
import numpy as np
import pytest

from test_oracle_flow import _rand_cloud, _sympy_field


def test_field_at_particles_is_their_velocity(oracle):
    """Eq. 3 evaluated at q_i is dq_i/dt of Eq. 1 (F_i, the i = j term included)."""
    q, p = _rand_cloud(40, 3)
    v = oracle.velocity(q, p, q, 2.0)
    F, _, _ = oracle.rhs(q, p, 2.0)
    np.testing.assert_allclose(v, F, rtol=1e-14, atol=1e-15)


def test_tracers_on_particles_follow_them(oracle):
    q, p = _rand_cloud(30, 4)
    x0 = np.concatenate([q[::3], q[7:8]])
    q1, p1, x1 = oracle.flow(q, p, x0, 1.5, 12)
    q1r, p1r, _ = oracle.shoot(q, p, 1.5, 12)
    assert np.array_equal(q1, q1r) and np.array_equal(p1, p1r)
    np.testing.assert_allclose(x1, np.concatenate([q1[::3], q1[7:8]]), rtol=1e-13, atol=1e-13)


def test_far_tracer_does_not_move(oracle):
    """G underflows to 0 beyond ~38.6 sigma in FP64: a tracer 100 sigma away stays put."""
    q, p = _rand_cloud(20, 5, scale=1.0)
    x0 = np.array([[300.0, 0.0, 0.0], [0.0, -250.0, 90.0]])
    _, _, x1 = oracle.flow(q, p, x0, 1.0, 9)
    assert np.array_equal(x1, x0)


def test_field_is_linear_in_momentum(oracle):
    q, p = _rand_cloud(25, 6)
    x = np.random.default_rng(1).normal(scale=3.0, size=(17, 3))
    v1 = oracle.velocity(q, p, x, 1.3)
    v2 = oracle.velocity(q, 2.0 * p, x, 1.3)
    assert np.array_equal(v2, 2.0 * v1)
    assert np.array_equal(oracle.velocity(q, np.zeros_like(p), x, 1.3), np.zeros_like(x))


def test_single_particle_closed_form(oracle):
    """N = 1: the particle moves as q0 + t p0 (F = p0, Phi = 0), so the tracer's
    Euler recurrence is x <- x + h exp(-|x - q0 - k h p0|^2 / (2 sigma^2)) p0."""
    q0 = np.array([[0.5, -1.0, 2.0]])
    p0 = np.array([[0.8, 0.3, -0.4]])
    x0 = np.array([[1.0, -0.5, 2.5], [-2.0, 0.0, 1.0]])
    sigma, T = 1.2, 16
    _, _, x1 = oracle.flow(q0, p0, x0, sigma, T)
    h = 1.0 / T
    x = x0.copy()
    qk = q0[0].copy()
    for _ in range(T):
        g = np.exp(-np.sum((x - qk) ** 2, axis=1) / (2 * sigma ** 2))
        x = x + h * g[:, None] * p0[0][None, :]
        qk = qk + h * p0[0]
    np.testing.assert_allclose(x1, x, rtol=1e-13, atol=1e-14)


def test_tracer_euler_converges_to_dop853(oracle):
    """Particles and tracers integrated as one ODE system by an 8th-order
    integrator (symbolic field): the Euler tracers' error shrinks like h."""
    integ = pytest.importorskip("scipy.integrate")
    sp = pytest.importorskip("sympy")
    n, m, sigma = 3, 2, 1.0
    field, _ = _sympy_field(n, sigma)
    qs = sp.symbols(f"q0:{3 * n}")
    ps = sp.symbols(f"p0:{3 * n}")
    xs = sp.symbols("x0:3")
    vel = [sum(sp.exp(-sum((xs[a] - qs[3 * i + a]) ** 2 for a in range(3)) / (2 * sigma ** 2))
               * ps[3 * i + c] for i in range(n)) for c in range(3)]
    fv = sp.lambdify(list(qs) + list(ps) + list(xs), vel, "math")
    rng = np.random.default_rng(8)
    q0 = rng.normal(scale=0.8, size=(n, 3))
    p0 = rng.normal(scale=0.5, size=(n, 3))
    x0 = rng.normal(scale=1.0, size=(m, 3))

    def f(_t, y):
        q, p, x = y[:3 * n].reshape(n, 3), y[3 * n:6 * n].reshape(n, 3), y[6 * n:].reshape(m, 3)
        a, b = field(q, p)
        args = list(q.ravel()) + list(p.ravel())
        v = np.array([fv(*(args + list(x[k]))) for k in range(m)])
        return np.concatenate([a.ravel(), b.ravel(), v.ravel()])

    y0 = np.concatenate([q0.ravel(), p0.ravel(), x0.ravel()])
    sol = integ.solve_ivp(f, (0.0, 1.0), y0, method="DOP853", rtol=1e-13, atol=1e-13)
    x_true = sol.y[6 * n:, -1].reshape(m, 3)
    errs = [np.abs(oracle.flow(q0, p0, x0, sigma, T)[2] - x_true).max() for T in (50, 100, 200)]
    ratios = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_tracers_translation_equivariant(oracle):
    q, p = _rand_cloud(15, 9)
    x0 = np.random.default_rng(2).normal(scale=3.0, size=(11, 3))
    c = np.array([12.5, -40.0, 3.25])
    _, _, x1 = oracle.flow(q, p, x0, 1.7, 8)
    _, _, x1c = oracle.flow(q + c, p, x0 + c, 1.7, 8)
    np.testing.assert_allclose(x1c - c, x1, rtol=0, atol=1e-12)


def test_bh_field_at_particles_is_their_bh_velocity(oracle):
    """A tracer at a particle's position takes that particle's Barnes-Hut
    decisions (same FP32 position) and sums: v_BH(q_i) = F_BH,i exactly;
    Barnes-Hut tracers on particles follow them."""
    from paper_1907_04834_gb300 import inputs
    w = inputs.make("blobs", 600, 41)
    v = oracle.velocity(w.q0, w.p0, w.q0, w.sigma, mode=oracle.BH)
    F, _, _ = oracle.rhs(w.q0, w.p0, w.sigma, mode=oracle.BH)
    assert np.array_equal(v, F)
    x0 = w.q0[::4].copy()
    q1, _, x1 = oracle.flow(w.q0, w.p0, x0, w.sigma, 6, mode=oracle.BH)
    assert np.array_equal(x1, q1[::4])


def test_bh_field_limits_and_linearity(oracle):
    from paper_1907_04834_gb300 import inputs
    w = inputs.make("blobs", 500, 42)
    rng = np.random.default_rng(3)
    x = w.q0[rng.choice(500, 40)] + rng.normal(scale=2.0, size=(40, 3))
    ve = oracle.velocity(w.q0, w.p0, x, w.sigma)
    vinf = oracle.velocity(w.q0, w.p0, x, w.sigma, mode=oracle.BH, thresh=1e30)
    np.testing.assert_allclose(vinf, ve, rtol=1e-12, atol=1e-15 * np.abs(ve).max())
    v1 = oracle.velocity(w.q0, w.p0, x, w.sigma, mode=oracle.BH)
    v2 = oracle.velocity(w.q0, 2.0 * w.p0, x, w.sigma, mode=oracle.BH)
    assert np.array_equal(v2, 2.0 * v1)
    assert np.abs(v1 - ve).max() <= 0.05 * np.abs(ve).max()  # approximation, not garbage
