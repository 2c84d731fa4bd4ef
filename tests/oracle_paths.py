"""The oracle's Euler steps and discrete adjoint (Sec. 2.1, Eq. 1-2; Sec. 2.2
in Barnes-Hut mode) taken along a given discrete path -- the oracle's own, or
the CUDA path's -- written with the oracle's right-hand sides as numpy loops
in the oracle's update order (test helpers, no test cases here).

The Barnes-Hut map is discontinuous: two paths that differ by rounding can
take different decisions for a target whose distance to a node sits at the
threshold, and then part by more than rounding.  Evaluating the oracle on the
CUDA path's own states compares the two implementations step by step on
shared states, where their decisions must agree exactly."""
import numpy as np


def euler_path(oracle, q0, p0, sigma, T, mode):
    """States (T + 1, N, 3) of the oracle's explicit Euler shooting."""
    h = 1.0 / T
    qs, ps = [q0.copy()], [p0.copy()]
    for _ in range(T):
        F, Phi, _ = oracle.rhs(qs[-1], ps[-1], sigma, mode=mode)
        qs.append(qs[-1] + h * F)
        ps.append(ps[-1] + h * Phi)
    return np.stack(qs), np.stack(ps)


def step_residual(oracle, qs, ps, sigma, mode):
    """Largest |state k+1 - (state k + h * oracle RHS at state k)| over the
    steps of a given path, for q and for p."""
    T = len(qs) - 1
    h = 1.0 / T
    rq = rp = 0.0
    for k in range(T):
        F, Phi, _ = oracle.rhs(qs[k], ps[k], sigma, mode=mode)
        rq = max(rq, float(np.abs(qs[k + 1] - (qs[k] + h * F)).max()))
        rp = max(rp, float(np.abs(ps[k + 1] - (ps[k] + h * Phi)).max()))
    return rq, rp


def grad_on_path(oracle, qs, ps, X, sigma, lam, mode):
    """Objective (Eq. 2) and its discrete-adjoint gradient with respect to
    p0 with every step's right-hand sides taken at the given path's states:
    E = [E, H(q0, p0), lambda |q_T - X|^2], grad."""
    T = len(qs) - 1
    h = 1.0 / T
    F0, _, _ = oracle.rhs(qs[0], ps[0], sigma, mode=mode)
    H0 = 0.5 * float(np.sum(ps[0] * F0))
    data = lam * float(np.sum((qs[T] - X) ** 2))
    al = 2.0 * lam * (qs[T] - X)
    be = np.zeros_like(al)
    for k in range(T - 1, -1, -1):
        dA, dB, _ = oracle.adj_rhs(qs[k], ps[k], al, be, sigma, mode=mode)
        al = al + h * dA
        be = be + h * dB
    return np.array([H0 + data, H0, data]), be + F0
