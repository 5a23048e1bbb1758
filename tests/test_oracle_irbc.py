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


# --------------------------------------------------------------------------
# non-smooth model (irreversible investment, eq. modelkink1)
# --------------------------------------------------------------------------

def _irr_policy(I, N, mu_fn, sigma_pert=0.0):
    """Policy (k', mu, lambda) over x = (a, k): k' = k + a small seeded
    perturbation, lambda = lambda*, mu = mu_fn(k, a) on the (k_j, a_j) pairs."""
    lam = I.steady_lambda()
    d, m = 2 * N, 2 * N + 1

    def fn(dims, X):
        X = np.asarray(X, np.float64).reshape(-1, len(dims)) if len(dims) else np.zeros((np.atleast_2d(X).shape[0], 0))
        full = np.ones((X.shape[0], d))
        if len(dims):
            full[:, list(dims)] = X
        y = np.zeros((X.shape[0], m))
        y[:, :N] = full[:, N:] + sigma_pert * np.sin(5 * (full[:, :N] - 1))
        y[:, N:2 * N] = mu_fn(full[:, N:], full[:, :N])
        y[:, 2 * N] = lam
        # cut-HDMR: keep only the part living on `dims` (anchor contributions are exact here)
        return y

    E = O.OracleDDSG(d, m, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in [()] + [(i,) for i in range(d)] + [(j, N + j) for j in range(N)]:
        E.add_regular(u, 4)
    E.fill_values(fn)
    E.hierarchize()
    return E, lam


def test_fischer_burmeister_rows():
    """Row N + j is FB(mu_j, k'_j - (1 - delta) k_j) = mu + I - sqrt(mu^2 + I^2):
    zero on the complementarity set, 2 at (mu, I) = (3, 4)... scaled to the
    chosen guesses."""
    N = 2
    I = O.IRBCOracle(N, irreversible=True)
    E, lam = _irr_policy(I, N, lambda k, a: 0.0 * k)
    s = np.ones((1, 2 * N))
    dl = I.p["delta"]
    for mu, inv, want in ((0.0, 0.02, 0.0), (0.5, 0.0, 0.0), (0.03, 0.04, 0.02), (0.0, -0.01, -0.02)):
        g = np.concatenate([np.full(N, (1 - dl) + inv), np.full(N, mu), [lam]])[None]
        r = I.residual(E, s, g)[0]
        assert np.allclose(r[N:2 * N], want, atol=1e-15), (mu, inv, r[N:2 * N])


def test_irreversible_reduces_to_smooth_when_mu_vanishes():
    """With mu == 0 in the policy and the guess, the Euler rows of eq. modelkink1
    are those of eq. model1 and the resource row is eq. model2."""
    N = 3
    Ii = O.IRBCOracle(N, irreversible=True)
    Is = O.IRBCOracle(N)
    E, lam = _irr_policy(Ii, N, lambda k, a: 0.0 * k, sigma_pert=0.01)
    Es = O.OracleDDSG(2 * N, N + 1, lo=np.full(2 * N, 0.8), hi=np.full(2 * N, 1.2))
    for c, u in enumerate(E.comps):
        cs = Es.add_component(u, E.lv[c], E.ix[c])
        Es.set_values(cs, E.values[c][:, list(range(N)) + [2 * N]])
    Es.hierarchize()
    rng = np.random.default_rng(4)
    S = 0.9 + 0.2 * rng.random((5, 2 * N))
    gk = S[:, N:] * (1 + 0.01 * rng.random((5, N)))
    gi = np.concatenate([gk, np.zeros((5, N)), np.full((5, 1), lam)], 1)
    gs = np.concatenate([gk, np.full((5, 1), lam)], 1)
    for form in (0, 1):
        ri, ei = Ii.residual(E, S, gi, form=form, want_err=True)
        rs, es = Is.residual(Es, S, gs, form=form, want_err=True)
        assert np.allclose(ri[:, :N], rs[:, :N], rtol=1e-12, atol=1e-13)
        assert np.allclose(ri[:, 2 * N], rs[:, N], rtol=1e-12, atol=1e-13)
        assert np.allclose(ei, es, rtol=1e-12, atol=1e-14)


def test_irreversible_steady_state_and_newton():
    """sigma = 0, a = k = 1: (k' = 1, mu = 0, lambda*) zeroes every row
    (investment delta > 0, so the constraint is slack); Newton from a perturbed
    guess returns there, and from a state whose capital must shrink it lands on
    the constraint: k' = (1 - delta) k with mu > 0."""
    N = 2
    I = O.IRBCOracle(N, irreversible=True, sigma=0.0)
    E, lam = _irr_policy(I, N, lambda k, a: 0.0 * k)
    s = np.ones((1, 2 * N))
    g = np.concatenate([np.ones(N), np.zeros(N), [lam]])[None]
    assert np.max(np.abs(I.residual(E, s, g)[0])) < 1e-12
    g0 = np.concatenate([[1.03, 0.98], [0.01, 0.0], [lam * 1.05]])[None]
    sol, _, nrm = I.newton(E, s, g0)
    assert nrm[0] < 1e-10 and np.allclose(sol[0], g[0], atol=1e-8)
    # a continuation policy that returns capital to 1 (k' = 1 everywhere): a
    # country holding k = 1.19 wants to disinvest faster than depreciation
    const = lambda dims, X: np.tile(np.concatenate([np.ones(N), np.zeros(N), [lam]]), (np.atleast_2d(X).shape[0], 1))
    E1 = O.OracleDDSG(2 * N, 2 * N + 1, lo=np.full(2 * N, 0.8), hi=np.full(2 * N, 1.2))
    for u in [()] + [(i,) for i in range(2 * N)] + [(j, N + j) for j in range(N)]:
        E1.add_regular(u, 3)
    E1.fill_values(const)
    E1.hierarchize()
    dl = I.p["delta"]
    for s2 in ([1.0, 1.0, 1.19, 1.0], [0.8, 1.0, 1.2, 1.0]):
        s2 = np.array([s2])
        sol2, _, nrm2 = I.newton(E1, s2, np.concatenate([[s2[0, 2], 1.0], [0.0, 0.0], [lam]])[None])
        assert nrm2[0] < 1e-10
        inv = sol2[0, :N] - (1 - dl) * s2[0, N:]
        mu = sol2[0, N:2 * N]
        assert np.all(inv > -1e-10) and np.all(mu > -1e-10) and np.all(np.abs(inv * mu) < 1e-10)
        assert mu[0] > 1e-3 and abs(inv[0]) < 1e-10      # country 0 sits on the constraint
        assert mu[1] == 0.0 and inv[1] > 1e-3            # country 1 invests
