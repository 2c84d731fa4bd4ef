"""Pins for the oracle's backward stage (discrete adjoint of the Euler map,
Sec. 2.1-2.2): central finite differences of the objective, the transpose
identity of one linearised step, and the lambda = 0 closed form."""
import numpy as np
import pytest

from paper_1907_04834_gb300 import inputs


def test_gradient_matches_central_differences(oracle):
    """dE/dp0 from the adjoint against central differences of E along random
    unit directions (the differences call only the forward shooting)."""
    w = inputs.make("slab", 120, 21, T=6)
    lam = 1.0
    E, g, _ = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, lam)
    rng = np.random.default_rng(2)
    for _ in range(8):
        v = rng.normal(size=w.p0.shape)
        v /= np.linalg.norm(v)
        eps = 1e-5 * max(1.0, np.abs(w.p0).max())
        Ep, _, _ = oracle.shoot_grad(w.q0, w.p0 + eps * v, w.X, w.sigma, w.T, lam)
        Em, _, _ = oracle.shoot_grad(w.q0, w.p0 - eps * v, w.X, w.sigma, w.T, lam)
        fd = (Ep[0] - Em[0]) / (2 * eps)
        an = float(np.sum(g * v))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.linalg.norm(g)), (fd, an)


def test_one_step_transpose_identity(oracle):
    """<J v, u> = <v, J^T u> for one Euler step (q,p) -> (q + hF, p + hPhi):
    J v by central differences of the forward step, J^T u from the adjoint
    right-hand side with (alpha, beta) = u."""
    rng = np.random.default_rng(4)
    n, sigma, h = 40, 1.2, 0.25
    q = rng.normal(scale=2.0, size=(n, 3))
    p = rng.normal(scale=0.4, size=(n, 3))

    def step(qq, pp):
        F, Phi, _ = oracle.rhs(qq, pp, sigma)
        return qq + h * F, pp + h * Phi

    for _ in range(4):
        vq, vp = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
        uq, up = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
        eps = 1e-6
        a1, b1 = step(q + eps * vq, p + eps * vp)
        a0, b0 = step(q - eps * vq, p - eps * vp)
        Jv_q, Jv_p = (a1 - a0) / (2 * eps), (b1 - b0) / (2 * eps)
        lhs = float(np.sum(Jv_q * uq) + np.sum(Jv_p * up))
        dA, dB, _ = oracle.adj_rhs(q, p, uq, up, sigma)
        JTu_q, JTu_p = uq + h * dA, up + h * dB
        rhs = float(np.sum(vq * JTu_q) + np.sum(vp * JTu_p))
        assert lhs == pytest.approx(rhs, rel=1e-8)


def test_zero_lambda_gradient_is_Kp(oracle):
    """With lambda = 0, E = H(q0,p0) and dE/dp0 = K(q0) p0 = F(q0,p0)."""
    w = inputs.make("blobs", 300, 8, T=4)
    E, g, _ = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, 0.0)
    F, _, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    np.testing.assert_allclose(g, F, rtol=0, atol=1e-15 * np.abs(F).max())
    assert E[2] == 0.0


def test_adjoint_rows_match_full(oracle):
    w = inputs.make("slab", 90, 3, T=2)
    rng = np.random.default_rng(1)
    al, be = rng.normal(size=w.q0.shape), rng.normal(size=w.q0.shape)
    dA, dB, _ = oracle.adj_rhs(w.q0, w.p0, al, be, w.sigma)
    rows = np.array([0, 7, 89, 45])
    rA, rB = oracle.adj_rhs_rows(w.q0, w.p0, al, be, w.sigma, rows)
    assert np.array_equal(rA, dA[rows]) and np.array_equal(rB, dB[rows])
    F, Phi, _ = oracle.rhs(w.q0, w.p0, w.sigma)
    rF, rP = oracle.rhs_rows(w.q0, w.p0, w.sigma, rows)
    assert np.array_equal(rF, F[rows]) and np.array_equal(rP, Phi[rows])


def test_adjoint_along_a_given_path_is_the_oracles(oracle):
    """The numpy step and adjoint loops of the path helpers reproduce the
    oracle's own shooting and gradient on its own path: states bit for bit,
    the gradient bit for bit, E to summation order (exact and Barnes-Hut)."""
    from oracle_paths import euler_path, grad_on_path, step_residual
    w = inputs.make("blobs", 400, 33, T=5)
    for mode in (oracle.EXACT, oracle.BH):
        qs, ps = euler_path(oracle, w.q0, w.p0, w.sigma, w.T, mode)
        q1, p1, _ = oracle.shoot(w.q0, w.p0, w.sigma, w.T, mode=mode)
        assert np.array_equal(qs[-1], q1) and np.array_equal(ps[-1], p1)
        assert step_residual(oracle, qs, ps, w.sigma, mode) == (0.0, 0.0)
        E, g = grad_on_path(oracle, qs, ps, w.X, w.sigma, w.lam, mode)
        Eo, go, _ = oracle.shoot_grad(w.q0, w.p0, w.X, w.sigma, w.T, w.lam, mode=mode)
        assert np.array_equal(g, go)
        np.testing.assert_allclose(E, Eo, rtol=1e-13)
