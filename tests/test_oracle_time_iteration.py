"""Pins of the oracle's adaptive DDSG time iteration (Alg. 1 around Alg. 2):

- eq. 3.18 / 3.19 against closed forms: for f = 1 + |x0-1||x1-1| on [0.8,1.2]^3
  every grid is exact, so the component integrals are Q f_empty = 1, Q f_i = 0,
  Q f_01 = 0.16 * (1/4)^2 = 0.01 and Q f_02 = Q f_12 = 0: eta_01 = 0.01,
  eta_02 = eta_12 = 0, rho = (0, 0.01); pruning drops the zero pairs.
- one time-iteration step solves the Euler equations at every grid node: the
  new policy, evaluated at the cut states of its grids, has residual ~0 under
  the previous policy (node reproduction of the cut-HDMR interpolant).
- the iteration improves the Euler errors at fresh states."""
import numpy as np

import oracle as O
import synth
from oracle.time_iteration import oracle_build_ddsg, oracle_solver, oracle_time_iteration


def _abs_product(X):
    X = np.atleast_2d(X)
    return np.stack([1.0 + np.abs(X[:, 0] - 1.0) * np.abs(X[:, 1] - 1.0),
                     2.0 - 0.5 * np.abs(X[:, 0] - 1.0) * np.abs(X[:, 1] - 1.0)], 1)


def test_eta_rho_closed_forms():
    d, m = 3, 2
    # eps_eta < 0 keeps every pair (a pair is kept iff eta > eps_eta)
    E, info = oracle_build_ddsg(_abs_product, d, m, 2, 3, -1.0, -1.0, 0.0, np.full(d, 0.8), np.full(d, 1.2))
    assert len(info["components"]) == 1 + 3 + 3
    assert abs(info["eta"][(0, 1)] - 0.01 * np.sqrt(1 + 0.25) / np.sqrt(1 + 4)) < 1e-14
    assert info["eta"][(0, 2)] < 1e-15 and info["eta"][(1, 2)] < 1e-15
    assert info["rho"][0] < 1e-15
    assert abs(info["rho"][1] - info["eta"][(0, 1)]) < 1e-14
    E2, info2 = oracle_build_ddsg(_abs_product, d, m, 2, 3, -1.0, 1e-6, 0.0, np.full(d, 0.8), np.full(d, 1.2))
    assert info2["components"] == [(), (0,), (1,), (2,), (0, 1)]
    assert sorted(info2["rejected"]) == [(0, 2), (1, 2)]
    X = synth.uniform_matrix(3, 50, d, 0.8, 1.2)
    assert np.allclose(E2.eval(X, form=1)["y"], _abs_product(X), atol=1e-14)


def _initial_policy(I, N):
    lam = I.steady_lambda()
    d = 2 * N

    def fn(dims, X):
        y = np.tile(np.concatenate([np.ones(N), [lam]]), (X.shape[0], 1))
        for a, dim in enumerate(dims):
            if dim >= N:
                y[:, dim - N] = X[:, a]
        return y

    E = O.OracleDDSG(d, N + 1, lo=np.full(d, 0.8), hi=np.full(d, 1.2))
    for u in [()] + [(i,) for i in range(d)]:
        E.add_regular(u, 2)
    E.fill_values(fn)
    E.hierarchize()
    return E


def test_step_solves_the_euler_equations_at_every_node():
    N = 2
    d = 2 * N
    I = O.IRBCOracle(N)
    E0 = _initial_policy(I, N)
    lo, hi = np.full(d, 0.8), np.full(d, 1.2)
    E1, info = oracle_build_ddsg(oracle_solver(I, E0), d, N + 1, 2, 3, -1.0, -1.0, 0.0, lo, hi)
    for c, u in enumerate(E1.comps):
        S = np.tile(0.5 * (lo + hi), (E1.npts(c), 1))
        if u:
            S[:, list(u)] = E1.node_coords_phys(c)
        g = E1.eval(S, form=1)["y"]
        r = I.residual(E0, S, g, form=1)
        assert np.max(np.abs(r)) < 1e-8, (u, np.max(np.abs(r)))


def test_time_iteration_improves_euler_errors():
    N = 2
    d = 2 * N
    I = O.IRBCOracle(N)
    E0 = _initial_policy(I, N)
    T = synth.irbc_states(synth.BASE_SEED + 600, 40, N)
    g0 = E0.eval(T, form=1)["y"]
    _, e0 = I.residual(E0, T, g0, form=1, want_err=True)
    pairs = lambda k: [(i,) for i in range(d)] if k == 1 else [(j, N + j) for j in range(N)]
    _, hist = oracle_time_iteration(I, E0, 3, 2, 4, 1e-4, -1.0, 0.0, np.full(d, 0.8), np.full(d, 1.2), T,
                                    candidates=pairs)
    errs = [h["euler_error_mean"] for h in hist]
    assert errs[-1] < errs[0] < float(np.mean(np.max(e0, 1)))
