"""Pins for the oracle's semi-implicit symplectic Euler shooting (a variant of
the time discretisation of Sec. 2.1): zero fixed-point passes give explicit
Euler; with many passes one step solves the implicit symplectic Euler
equations (solved here independently on the symbolic field) and the step map
is symplectic; trajectories converge at first order."""
import numpy as np
import pytest

from test_oracle_flow import _rand_cloud, _sympy_field


def test_zero_passes_is_explicit_euler(oracle):
    q, p = _rand_cloud(25, 11)
    a = oracle.shoot(q, p, 1.7, 9)
    b = oracle.shoot_sympl(q, p, 1.7, 9, 0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    from paper_1907_04834_gb300 import inputs
    w = inputs.make("blobs", 400, 5)
    a = oracle.shoot(w.q0, w.p0, w.sigma, 4, mode=oracle.BH)
    b = oracle.shoot_sympl(w.q0, w.p0, w.sigma, 4, 0, mode=oracle.BH)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_step_solves_implicit_equations(oracle):
    """One step (T = 1/h) with many passes equals the solution of
    p1 = p0 + h Phi(q0, p1), q1 = q0 + h F(q0, p1) found by a root finder on
    the symbolically differentiated field."""
    opt = pytest.importorskip("scipy.optimize")
    n, sigma, h = 3, 1.0, 0.25
    field, _ = _sympy_field(n, sigma)
    rng = np.random.default_rng(3)
    q0 = rng.normal(scale=0.8, size=(n, 3))
    p0 = rng.normal(scale=0.4, size=(n, 3))

    def resid(pf):
        p1 = pf.reshape(n, 3)
        _, Phi = field(q0, p1)
        return (p1 - p0 - h * Phi).ravel()

    p1 = opt.fsolve(resid, p0.ravel(), xtol=1e-14).reshape(n, 3)
    F, Phi = field(q0, p1)
    q_ref, p_ref = q0 + h * F, p0 + h * Phi
    # F is linear and Phi quadratic in p, so one step of size h from (q0, p0)
    # is one step of size 1 (T = 1) from (q0, h p0), with p scaled by h
    q1, pp1, _ = oracle.shoot_sympl(q0, h * p0, sigma, 1, 60)
    np.testing.assert_allclose(q1, q_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pp1 / h, p_ref, rtol=0, atol=1e-12)


def test_converged_step_is_symplectic(oracle):
    """The converged step map (q0, p0) -> (q1, p1) preserves the symplectic
    form: J^T Omega J = Omega (finite-difference Jacobian); explicit Euler
    does not."""
    n, sigma, T = 2, 1.0, 4
    rng = np.random.default_rng(9)
    q0 = rng.normal(scale=0.7, size=(n, 3))
    p0 = rng.normal(scale=0.5, size=(n, 3))
    d = 6 * n

    def step(z, iters):
        q1, p1, _ = oracle.shoot_sympl(z[:3 * n].reshape(n, 3), z[3 * n:].reshape(n, 3),
                                       sigma, T, iters)
        return np.concatenate([q1.ravel(), p1.ravel()])

    z0 = np.concatenate([q0.ravel(), p0.ravel()])
    Om = np.block([[np.zeros((3 * n, 3 * n)), np.eye(3 * n)],
                   [-np.eye(3 * n), np.zeros((3 * n, 3 * n))]])

    def defect(iters):
        eps = 1e-6
        J = np.empty((d, d))
        for k in range(d):
            e = np.zeros(d)
            e[k] = eps
            J[:, k] = (step(z0 + e, iters) - step(z0 - e, iters)) / (2 * eps)
        return np.abs(J.T @ Om @ J - Om).max()

    assert defect(80) < 1e-7
    assert defect(0) > 1e-3


def test_sympl_converges_to_dop853(oracle):
    integ = pytest.importorskip("scipy.integrate")
    n, sigma = 3, 1.0
    field, _ = _sympy_field(n, sigma)
    rng = np.random.default_rng(7)
    q0 = rng.normal(scale=0.8, size=(n, 3))
    p0 = rng.normal(scale=0.5, size=(n, 3))

    def f(_t, y):
        a, b = field(y[: 3 * n].reshape(n, 3), y[3 * n:].reshape(n, 3))
        return np.concatenate([a.ravel(), b.ravel()])

    sol = integ.solve_ivp(f, (0.0, 1.0), np.concatenate([q0.ravel(), p0.ravel()]),
                          method="DOP853", rtol=1e-13, atol=1e-13)
    q_true = sol.y[: 3 * n, -1].reshape(n, 3)
    errs = [np.abs(oracle.shoot_sympl(q0, p0, sigma, T, 30)[0] - q_true).max()
            for T in (50, 100, 200)]
    ratios = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_gradient_zero_passes_is_explicit_gradient(oracle):
    """The semi-implicit scheme's gradient with no passes is the explicit
    scheme's, bit for bit (exact and Barnes-Hut)."""
    from paper_1907_04834_gb300 import inputs
    w = inputs.make("blobs", 300, 6, T=5)
    for mode in (oracle.EXACT, oracle.BH):
        a = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=mode)
        b = oracle.shoot_grad_sympl(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, 0, mode=mode)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("M", [1, 2, 4])
def test_gradient_matches_finite_differences(oracle, M):
    """Central differences of the objective E(p0) = H(q0, p0) + lambda |q(1) -
    X|^2 of the semi-implicit shooting (forward map of shoot_sympl, FP64)
    along random directions against the adjoint gradient; strongly moving
    points (momenta of several sigma per unit time) so the passes matter."""
    q, p = _rand_cloud(40, 21 + M)
    p = 3.0 * p
    sigma, T, lam = 1.3, 6, 0.7
    X = q + np.random.default_rng(M).normal(scale=0.5, size=q.shape)
    E, g, q1 = oracle.shoot_grad_sympl(q, p, X, sigma, T, lam, M)
    q1s, _, H = oracle.shoot_sympl(q, p, sigma, T, M)
    assert np.array_equal(q1, q1s)
    assert abs(E[0] - (H[0] + lam * np.sum((q1s - X) ** 2))) <= 1e-12 * abs(E[0])

    def Eof(pp):
        qq, _, HH = oracle.shoot_sympl(q, pp, sigma, T, M)
        return HH[0] + lam * np.sum((qq - X) ** 2)

    rng = np.random.default_rng(100 + M)
    eps = 1e-5
    for _ in range(6):
        v = rng.normal(size=p.shape)
        v /= np.linalg.norm(v)
        fd = (Eof(p + eps * v) - Eof(p - eps * v)) / (2 * eps)
        d = float(np.sum(g * v))
        assert abs(fd - d) <= 1e-6 * np.linalg.norm(g), (fd, d)
    # the passes change the gradient: it is not the explicit scheme's
    _, g0, _ = oracle.shoot_grad(q, p, X, sigma, T, lam)
    assert np.linalg.norm(g - g0) > 1e-4 * np.linalg.norm(g0)
