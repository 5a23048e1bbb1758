"""Seeded synthetic inputs shared by the CUDA path, its tests and the CPU oracle.

This module holds NO arithmetic of the DDSG method (no basis functions, no
surpluses, no HDMR combination, no IRBC equations). It only draws numbers and
evaluates the *functions being approximated* (the kinked test family, the
synthetic IRBC policy used as grid values), so that both sides of a parity test
see bit-identical inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output k of stream `seed` is
mix(seed + (k+1)*0x9E3779B97F4A7C15), and a 53-bit uniform is (z >> 11)*2^-53.
Seeds are 20220214 + a workload id.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
BASE_SEED = 20220214

# workload ids (added to BASE_SEED)
W_SG4 = 1        # single regular sparse grid, d=4, level 5
W_D20 = 2        # cut-HDMR order 2, d=20
W_D100 = 3       # cut-HDMR order 2, d=100
W_IRBC150 = 4    # IRBC Euler residual sweep, N=150
W_IRBC20 = 5     # IRBC N=20 warm-start study


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 stream started at `seed`."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
    return _mix(s)


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0,1) with 53 random bits each."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_matrix(seed: int, rows: int, cols: int, lo=0.0, hi=1.0) -> np.ndarray:
    u = uniform(seed, rows * cols).reshape(rows, cols)
    return lo + (hi - lo) * u


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    u = uniform(seed, 2 * n).reshape(n, 2)
    u1 = np.maximum(u[:, 0], 2.0 ** -60)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u[:, 1])


# ---------------------------------------------------------------------------
# The kinked test family f_j(x) = exp(-sum_i c_ji (x_i - 1/2)^2) + 1/2 max(0, x_j - 0.7)
# on [0,1]^d, j = 0..m-1, c_ji ~ U[0.5, 2].
# ---------------------------------------------------------------------------

def family_coeffs(seed: int, m: int, d: int) -> np.ndarray:
    """c[j, i] ~ U[0.5, 2], shape (m, d)."""
    return uniform_matrix(seed + 1000, m, d, 0.5, 2.0)


def family_full(c: np.ndarray, x: np.ndarray) -> np.ndarray:
    """f(x) for full points x of shape (n, d); returns (n, m)."""
    x = np.asarray(x, dtype=np.float64)
    m = c.shape[0]
    q = ((x[:, None, :] - 0.5) ** 2 * c[None, :, :]).sum(axis=2)
    y = np.exp(-q)
    y += 0.5 * np.maximum(0.0, x[:, :m] - 0.7)
    return y


def family_cut(c: np.ndarray, dims, coords: np.ndarray) -> np.ndarray:
    """f at points whose coordinates outside `dims` sit at the anchor 1/2.

    coords has shape (n, len(dims)) and gives the coordinates on `dims`
    (canonical [0,1] units). With the other coordinates at 1/2 their quadratic
    terms vanish and their kink terms are max(0, 0.5-0.7) = 0, so this equals
    family_full on the assembled d-dim point; it just avoids building it.
    Returns (n, m).
    """
    coords = np.asarray(coords, dtype=np.float64)
    if coords.ndim == 1:
        coords = coords.reshape(-1, len(dims))
    m = c.shape[0]
    n = coords.shape[0]
    q = np.zeros((n, m))
    for a, dim in enumerate(dims):
        q += (coords[:, a:a + 1] - 0.5) ** 2 * c[None, :, dim]
    y = np.exp(-q)
    for a, dim in enumerate(dims):
        if dim < m:
            y[:, dim] += 0.5 * np.maximum(0.0, coords[:, a] - 0.7)
    return y


# ---------------------------------------------------------------------------
# Query sets
# ---------------------------------------------------------------------------

def uniform_queries(seed: int, n: int, d: int) -> np.ndarray:
    return uniform_matrix(seed + 2000, n, d)


def uniform_queries_rows(seed: int, lo: int, hi: int, d: int) -> np.ndarray:
    """Rows lo..hi-1 of uniform_queries(seed, n, d) for any n >= hi, drawn directly
    from their place in the stream (no prefix is generated)."""
    return uniform(seed + 2000, (hi - lo) * d, offset=lo * d).reshape(hi - lo, d)


def monomial_shaped_queries(seed: int, n_states: int, n_countries: int, s: float = 0.01):
    """States U[0,1]^(2N) (first N coordinates: productivity block, last N:
    capital block), each expanded into 2(N+1) shifted copies: copy +-i moves
    productivity coordinate i by +-s*sqrt(N+1); copy +-global moves all N
    productivity coordinates by +-s*sqrt(N+1). Shape (n_states*2(N+1), 2N).
    The result is NOT clamped to [0,1]: clamping is the evaluator's job."""
    N = n_countries
    d = 2 * N
    st = uniform_matrix(seed + 3000, n_states, d)
    h = s * math.sqrt(N + 1)
    nodes = []
    for i in range(N + 1):
        for sgn in (1.0, -1.0):
            sh = np.zeros(d)
            if i < N:
                sh[i] = sgn * h
            else:
                sh[:N] = sgn * h
            nodes.append(sh)
    nodes = np.array(nodes)  # (2(N+1), d)
    q = st[:, None, :] + nodes[None, :, :]
    return q.reshape(-1, d)


# ---------------------------------------------------------------------------
# IRBC workloads: states and a synthetic policy (grid values)
# ---------------------------------------------------------------------------

IRBC_LO = 0.8
IRBC_HI = 1.2


def irbc_states(seed: int, n: int, n_countries: int) -> np.ndarray:
    """n states (a_1..a_N, k_1..k_N) uniform in [0.8, 1.2]^(2N)."""
    return uniform_matrix(seed + 4000, n, 2 * n_countries, IRBC_LO, IRBC_HI)


def irbc_policy_perturbation(seed: int, n_countries: int):
    """Coefficients of a smooth seeded perturbation of the constant policy:
    returns (amp, freq, amp2): amp, freq of shape (N+1, 2N) with
    amp ~ U[-1,1]*1e-2/(2N), freq ~ U[0.5, 2]; amp2 of shape (N+1, N),
    ~ U[-1,1]*1e-2, weights of the pairwise terms in (a_j, k_j)."""
    N = n_countries
    amp = (uniform_matrix(seed + 5000, N + 1, 2 * N) * 2.0 - 1.0) * (1e-2 / (2 * N))
    freq = uniform_matrix(seed + 6000, N + 1, 2 * N, 0.5, 2.0)
    amp2 = (uniform_matrix(seed + 7000, N + 1, N) * 2.0 - 1.0) * 1e-2
    return amp, freq, amp2


def irbc_policy_values(base: np.ndarray, pert, dims, coords_phys: np.ndarray) -> np.ndarray:
    """Synthetic policy over x = (a_1..a_N, k_1..k_N):
        p(x) = base + sum_i amp[:, i] sin(freq[:, i] (x_i - 1))
                    + sum_j amp2[:, j] sin(8 (a_j - 1)) sin(8 (k_j - 1)),
    evaluated where only the coordinates `dims` differ from the anchor (x = 1
    there, so every other term vanishes). pert = (amp, freq, amp2) from
    irbc_policy_perturbation. coords_phys: (n, len(dims)). Returns (n, N+1)."""
    amp, freq, amp2 = pert
    N = amp2.shape[1]
    coords_phys = np.asarray(coords_phys, dtype=np.float64)
    if coords_phys.ndim == 1:
        coords_phys = coords_phys.reshape(-1, len(dims))
    n = coords_phys.shape[0]
    y = np.repeat(np.asarray(base, dtype=np.float64)[None, :], n, axis=0)
    for a, dim in enumerate(dims):
        y += amp[None, :, dim] * np.sin(freq[None, :, dim] * (coords_phys[:, a:a + 1] - 1.0))
    pos = {dim: a for a, dim in enumerate(dims)}
    for j in range(N):
        if j in pos and N + j in pos:
            y += amp2[None, :, j] * (np.sin(8.0 * (coords_phys[:, pos[j]:pos[j] + 1] - 1.0)) *
                                     np.sin(8.0 * (coords_phys[:, pos[N + j]:pos[N + j] + 1] - 1.0)))
    return y


def irbc_steady_lambda(gamma, tau, A: float, delta: float) -> float:
    """Multiplier of the deterministic steady state (a = k = k' = 1): the lambda
    solving sum_j (lambda / tau_j)^(-gamma_j) = N (A - delta), by bisection.
    Used as the base value of the synthetic policy."""
    gamma = np.asarray(gamma, np.float64)
    tau = np.asarray(tau, np.float64)
    target = gamma.size * (A - delta)
    lo, hi = 1e-8, 1e8
    for _ in range(400):
        mid = math.sqrt(lo * hi)
        if np.sum((mid / tau) ** (-gamma)) > target:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)
