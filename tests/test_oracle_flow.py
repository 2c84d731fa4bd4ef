"""Pins for the oracle's exact flow (Sec. 2.1, Eq. 1-2) against facts that do
not come from the oracle's own formulas: the Hamiltonian's automatic
derivatives, a high-order ODE integrator, closed forms, conservation laws and
symmetries."""
import math

import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs


def _rand_cloud(n, seed, scale=3.0, pscale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(scale=scale, size=(n, 3)), rng.normal(scale=pscale, size=(n, 3))


def _sympy_field(n, sigma):
    """Hamilton's vector field of H(q,p) = 1/2 sum_ij G(|q_i-q_j|) p_i.p_j
    (Sec. 2.1, Gaussian G(r) = exp(-r^2/(2 sigma^2))) by symbolic
    differentiation; returns callables dH/dp and -dH/dq and H."""
    sp = pytest.importorskip("sympy")
    q = sp.Matrix(sp.symbols(f"q0:{3 * n}")).reshape(n, 3)
    p = sp.Matrix(sp.symbols(f"p0:{3 * n}")).reshape(n, 3)
    H = 0
    for i in range(n):
        for j in range(n):
            r2 = sum((q[i, a] - q[j, a]) ** 2 for a in range(3))
            H += sp.exp(-r2 / (2 * sigma ** 2)) * sum(p[i, a] * p[j, a] for a in range(3))
    H = H / 2
    qs, ps = list(q), list(p)
    dHdp = [sp.diff(H, v) for v in ps]
    mdHdq = [-sp.diff(H, v) for v in qs]
    fp = sp.lambdify(qs + ps, dHdp, "math")
    fq = sp.lambdify(qs + ps, mdHdq, "math")
    fH = sp.lambdify(qs + ps, H, "math")

    def field(qv, pv):
        args = list(np.ravel(qv)) + list(np.ravel(pv))
        return (np.array(fp(*args)).reshape(n, 3), np.array(fq(*args)).reshape(n, 3))

    def ham(qv, pv):
        return float(fH(*(list(np.ravel(qv)) + list(np.ravel(pv)))))

    return field, ham


def test_rhs_is_hamiltons_vector_field(oracle):
    """F = dH/dp and Phi = -dH/dq (Eq. 1) with H the kinetic energy <p, K(q)p>/2."""
    n, sigma = 4, 1.7
    field, ham = _sympy_field(n, sigma)
    for seed in range(3):
        q, p = _rand_cloud(n, seed, scale=1.5)
        F, Phi, _ = oracle.rhs(q, p, sigma)
        Fs, Phis = field(q, p)
        np.testing.assert_allclose(F, Fs, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Phi, Phis, rtol=1e-12, atol=1e-14)
        # H(q0,p0) as reported by the shooting equals the symbolic Hamiltonian
        _, _, H = oracle.shoot(q, p, sigma, 3)
        assert H[0] == pytest.approx(ham(q, p), rel=1e-13)


def test_euler_converges_to_dop853(oracle):
    """Euler shooting error against an adaptive 8th-order integrator of the
    symbolic field shrinks like h (first order), to the integrator's limit."""
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
    errs = []
    for T in (50, 100, 200, 400):
        q1, _, _ = oracle.shoot(q0, p0, sigma, T)
        errs.append(np.abs(q1 - q_true).max())
    ratios = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)
    # Richardson extrapolation of a first-order method gains an order
    q100, _, _ = oracle.shoot(q0, p0, sigma, 100)
    q200, _, _ = oracle.shoot(q0, p0, sigma, 200)
    assert np.abs(2 * q200 - q100 - q_true).max() < errs[1] / 20


def test_single_point_closed_form(oracle):
    """N = 1: F = p (G(0) = 1), Phi = 0, so q(1) = q0 + p0, p(1) = p0."""
    q0 = np.array([[1.25, -3.5, 7.0]])
    p0 = np.array([[0.3, 0.1, -0.7]])
    for T in (1, 7, 10):
        q1, p1, H = oracle.shoot(q0, p0, 2.0, T)
        np.testing.assert_allclose(q1, q0 + p0, rtol=0, atol=1e-14)
        assert np.array_equal(p1, p0)
        assert H[0] == pytest.approx(0.5 * float(np.sum(p0 * p0)), rel=1e-15)


def test_far_clusters_move_independently(oracle):
    """Clusters 60 sigma apart do not interact: exp underflows to exactly 0,
    so shooting the union equals shooting each cluster alone, bit for bit."""
    sigma = 1.0
    qa, pa = _rand_cloud(20, 1, scale=1.0)
    qb, pb = _rand_cloud(15, 2, scale=1.0)
    qb = qb + np.array([60.0, 0.0, 0.0])
    qa1, pa1, _ = oracle.shoot(qa, pa, sigma, 5)
    qb1, pb1, _ = oracle.shoot(qb, pb, sigma, 5)
    q1, p1, _ = oracle.shoot(np.vstack([qa, qb]), np.vstack([pa, pb]), sigma, 5)
    assert np.array_equal(q1, np.vstack([qa1, qb1]))
    assert np.array_equal(p1, np.vstack([pa1, pb1]))


def test_total_momentum_conserved(oracle):
    """Phi is antisymmetric in (i, j): sum_i Phi_i = 0 and sum_i p_i is a
    constant of the discrete flow."""
    w = inputs.make("slab", 400, 11)
    F, Phi, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    scale = np.abs(Phi).sum()
    assert np.abs(Phi.sum(axis=0)).max() <= 1e-13 * scale
    _, p1, _ = oracle.shoot(w.q0, w.p0, w.sigma, 10)
    np.testing.assert_allclose(p1.sum(axis=0), w.p0.sum(axis=0), rtol=0,
                               atol=1e-13 * np.abs(w.p0).sum())


def test_hamiltonian_drift_is_first_order(oracle):
    """H is conserved by the exact flow; explicit Euler drifts by O(h)."""
    q0, p0 = _rand_cloud(60, 5, scale=2.0, pscale=0.4)
    drift = []
    for T in (20, 40, 80):
        _, _, H = oracle.shoot(q0, p0, 1.5, T)
        drift.append(abs(H[1] - H[0]))
    assert 1.8 < drift[0] / drift[1] < 2.2 and 1.8 < drift[1] / drift[2] < 2.2, drift


def test_equivariance(oracle):
    """Translation and rotation equivariance, permutation equivariance, and
    exact scaling (q, p, sigma) -> (2q, 2p, 2 sigma) => (2 q1, 2 p1)."""
    q0, p0 = _rand_cloud(50, 3)
    sigma, T = 2.0, 6
    q1, p1, _ = oracle.shoot(q0, p0, sigma, T)
    t = np.array([10.0, -4.0, 2.5])
    qt, pt, _ = oracle.shoot(q0 + t, p0, sigma, T)
    np.testing.assert_allclose(qt, q1 + t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pt, p1, rtol=0, atol=1e-12)
    rng = np.random.default_rng(0)
    Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    qr, pr, _ = oracle.shoot(q0 @ Rm.T, p0 @ Rm.T, sigma, T)
    np.testing.assert_allclose(qr, q1 @ Rm.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pr, p1 @ Rm.T, rtol=0, atol=1e-12)
    perm = rng.permutation(len(q0))
    qp, pp, _ = oracle.shoot(q0[perm], p0[perm], sigma, T)
    np.testing.assert_allclose(qp, q1[perm], rtol=0, atol=1e-13)
    np.testing.assert_allclose(pp, p1[perm], rtol=0, atol=1e-13)
    qs, ps, _ = oracle.shoot(2 * q0, 2 * p0, 2 * sigma, T)
    assert np.array_equal(qs, 2 * q1) and np.array_equal(ps, 2 * p1)


def test_small_momentum_linearisation(oracle):
    """q(1) - q0 = K(q0) p0 + O(|p0|^2), with K(q0)p0 = dH/dp from sympy."""
    n, sigma = 4, 1.3
    field, _ = _sympy_field(n, sigma)
    q0, p0 = _rand_cloud(n, 9, scale=1.2)
    Kp, _ = field(q0, p0)
    errs = []
    for eps in (1e-2, 5e-3):
        q1, _, _ = oracle.shoot(q0, eps * p0, sigma, 4)
        errs.append(np.abs((q1 - q0) / eps - Kp).max())
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.05)
    assert errs[1] < 1e-2 * np.abs(Kp).max()


def test_energy_terms(oracle):
    """E = H(q0,p0) + lambda |q(1) - X|^2 with the parts reported separately."""
    w = inputs.make("slab", 150, 4, T=5)
    E, _, q1 = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, 0.7)
    F, _, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    assert E[1] == pytest.approx(0.5 * float(np.sum(w.p0 * F)), rel=1e-14)
    assert E[2] == pytest.approx(0.7 * float(np.sum((q1 - w.X) ** 2)), rel=1e-14)
    assert E[0] == pytest.approx(E[1] + E[2], rel=1e-15)
    q1s, _, _ = oracle.shoot(w.q0, w.p0, w.sigma, w.T)
    assert np.array_equal(q1, q1s)


def test_angular_momentum(oracle):
    """H is rotation invariant, so the flow conserves L = sum_i q_i x p_i:
    the right-hand side satisfies sum_i (F_i x p_i + q_i x Phi_i) = 0 (Phi_ij
    along d_ij), and an Euler step changes L only by h^2 sum_i F_i x Phi_i, a
    drift that halves when T doubles."""
    q, p = _rand_cloud(50, 12, scale=1.5, pscale=0.5)
    F, Phi, _ = oracle.rhs(q, p, 1.2)
    r = (np.cross(F, p) + np.cross(q, Phi)).sum(axis=0)
    scale = np.abs(np.cross(F, p)).sum() + np.abs(np.cross(q, Phi)).sum()
    assert np.abs(r).max() <= 1e-13 * scale
    L0 = np.cross(q, p).sum(axis=0)
    drift = []
    for T in (20, 40, 80):
        q1, p1, _ = oracle.shoot(q, p, 1.2, T)
        drift.append(np.abs(np.cross(q1, p1).sum(axis=0) - L0).max())
    ratios = [drift[k] / drift[k + 1] for k in range(2)]
    assert all(1.8 < x < 2.2 for x in ratios), (drift, ratios)


def test_rk4_converges_at_fourth_order(oracle):
    """The right-hand side integrated by classical RK4 converges to an
    adaptive 8th-order solution of the symbolic field at fourth order (error
    ratio about 16 per halving of h): F and Phi are Hamilton's vector field to
    well below the Euler tests' resolution."""
    integ = pytest.importorskip("scipy.integrate")
    n, sigma = 3, 1.0
    field, _ = _sympy_field(n, sigma)
    rng = np.random.default_rng(17)
    q0 = rng.normal(scale=0.8, size=(n, 3))
    p0 = rng.normal(scale=0.6, size=(n, 3))

    def f(_t, y):
        a, b = field(y[: 3 * n].reshape(n, 3), y[3 * n:].reshape(n, 3))
        return np.concatenate([a.ravel(), b.ravel()])

    sol = integ.solve_ivp(f, (0.0, 1.0), np.concatenate([q0.ravel(), p0.ravel()]),
                          method="DOP853", rtol=1e-13, atol=1e-13)
    y_true = sol.y[:, -1]
    errs = []
    for T in (8, 16, 32):
        q1, p1 = oracle.shoot_rk4(q0, p0, sigma, T)
        errs.append(np.abs(np.concatenate([q1.ravel(), p1.ravel()]) - y_true).max())
    ratios = [errs[k] / errs[k + 1] for k in range(2)]
    assert all(13.0 < r < 19.0 for r in ratios), (errs, ratios)


def test_python_euler_loop_equals_shoot(oracle):
    """The step loop the GPU trajectory tests write in numpy (q += h F,
    p += h Phi with the oracle's right-hand side) is the oracle's own
    shooting, bit for bit, exact and Barnes-Hut."""
    w = inputs.make("blobs", 300, 31, T=5)
    for mode in (oracle.EXACT, oracle.BH):
        q, p = w.q0.copy(), w.p0.copy()
        h = 1.0 / w.T
        for _ in range(w.T):
            F, Phi, _ = oracle.rhs(q, p, w.sigma, mode=mode)
            q, p = q + h * F, p + h * Phi
        q1, p1, _ = oracle.shoot(w.q0, w.p0, w.sigma, w.T, mode=mode)
        assert np.array_equal(q, q1) and np.array_equal(p, p1)
