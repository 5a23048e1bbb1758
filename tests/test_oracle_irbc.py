"""Pins of the IRBC oracle (Sec. 2.1: eq. law_of_motion, model1, model2,
Table 1) against closed forms: Table 1 values, the monomial rule's moments,
the deterministic steady state, and the expectation of next-period
productivity under the rule at a = 1."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    out = {}
    for line in open(os.path.join(GOLD, "irbc_table1.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_table1_parameters():
    t = _table1()
    for key, v in t.items():
        assert O.IRBC_TABLE1[key] == v
    for N in (1, 2, 50, 150):
        I = O.IRBCOracle(N)
        b, a, dl = t["beta"], t["alpha"], t["delta"]
        # A is the deterministic steady-state rental condition: alpha beta A = 1 - beta (1 - delta)
        assert abs(a * b * I.A - (1 - b * (1 - dl))) < 1e-15
        assert abs(I.gamma[0] - 0.25) < 1e-15 and abs(I.gamma[-1] - (1.0 if N > 1 else 0.25)) < 1e-15
        assert np.all(np.abs(I.tau ** I.gamma - I.A) <= 1e-13 * I.A)


@pytest.mark.parametrize("n", [1, 2, 3, 11, 151])
def test_monomial_rule_moments(n):
    I = O.IRBCOracle(1)
    nodes, w = I.monomial(n)
    assert nodes.shape == (2 * n, n) and abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(w @ nodes, 0.0, atol=1e-14)                         # E[e] = 0
    assert np.allclose((nodes * w[:, None]).T @ nodes, np.eye(n), atol=1e-12)  # E[e e^T] = I
    for i, j, k in [(0, 0, 0), (0, min(1, n - 1), min(1, n - 1))]:
        assert abs(np.sum(w * nodes[:, i] * nodes[:, j] * nodes[:, k])) < 1e-12
    # degree-3 rule: exact for cubic polynomials, not for e_1^4 (true value 3)
    c = np.linspace(0.3, 1.1, n)
    f = lambda e: (e @ c) ** 2 + (e @ c) ** 3 + 2.0
    assert abs(np.sum(w * f(nodes)) - (c @ c + 2.0)) < 1e-11
    assert abs(np.sum(w * nodes[:, 0] ** 4) - n) < 1e-9


def _steady(N, sigma):
    I = O.IRBCOracle(N, sigma=sigma)
    lam = I.steady_lambda()
    const = np.concatenate([np.ones(N), [lam]])
    E = O.irbc_policy_ddsg(N, 3, lambda dims, X: np.repeat(const[None], X.shape[0], 0))
    return I, E, lam


@pytest.mark.parametrize("N", [1, 2, 5])
def test_deterministic_steady_state_zero_residual(N):
    I, E, lam = _steady(N, 0.0)
    # lambda* solves the resource constraint at k = k' = 1, a = 1
    assert abs(np.sum((lam / I.tau) ** (-I.gamma)) - N * (I.A - I.p["delta"])) < 1e-10
    s = np.ones((1, 2 * N))
    g = np.concatenate([np.ones(N), [lam]])[None]
    for form in (0, 1):
        r, ee = I.residual(E, s, g, form=form, want_err=True)
        assert np.max(np.abs(r)) < 1e-12
        assert np.max(ee) < 1e-12


@pytest.mark.parametrize("N", [2, 4])
def test_residual_expectation_of_productivity(N):
    """a = k = 1, constant policy (k'' = 1, lambda' = lambda*), sigma > 0: the
    only stochastic term is E[a'_j] over the 2(N+1) nodes, where a node moves
    a'_j iff it shocks country j or the global shock:
    E[a'_j] = 1 + (2 / (N+1)) (cosh(sigma sqrt(N+1)) - 1), so
    r_j = lambda* (1 - beta (1 - delta)) (1 - E[a'_j])."""
    sigma = 0.01
    I, E, lam = _steady(N, sigma)
    s = np.ones((1, 2 * N))
    g = np.concatenate([np.ones(N), [lam]])[None]
    r = I.residual(E, s, g)[0]
    Ea = 1.0 + (2.0 / (N + 1)) * (math.cosh(sigma * math.sqrt(N + 1)) - 1.0)
    ref = lam * (1.0 - I.p["beta"] * (1.0 - I.p["delta"])) * (1.0 - Ea)
    assert np.allclose(r[:N], ref, rtol=1e-9, atol=1e-15)
    assert abs(r[N]) < 1e-12     # resource constraint holds at the steady state


def test_newton_returns_to_the_steady_state():
    N = 3
    I, E, lam = _steady(N, 0.0)
    s = np.ones((1, 2 * N))
    g0 = np.concatenate([np.array([1.05, 0.97, 1.02]), [lam * 1.1]])[None]
    sol, its, norms = I.newton(E, s, g0)
    assert norms[0] < 1e-10 and its[0] >= 2
    assert np.allclose(sol[0], np.concatenate([np.ones(N), [lam]]), atol=1e-8)


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(9, 9)) + 3 * np.eye(9)
    b = rng.normal(size=9)
    x = b.copy()
    Ac = A.copy()
    assert O.lib().orc_lu_solve(9, O.ptr(Ac), O.ptr(x)) == 0
    assert np.allclose(A @ x, b, atol=1e-12)
    S = np.zeros((3, 3))
    assert O.lib().orc_lu_solve(3, O.ptr(S), O.ptr(np.ones(3))) == -1
