"""FP64 oracle of traces and diagonals of matrix functions from (L)DOS
moments (§6: centralities and connectivity indices written as traces and
diagonals of f(X); §2.1 operators, Eq. (5) shift and scale, Eq. (10)-(12)).

TEST INFRASTRUCTURE ONLY (see the package header).

With X~ = (X - c) / r holding the spectrum of X in [-1, 1] and f expanded as
f(c + r x) = sum_m g_m T_m(x) (the first coefficient carrying the 1/2 of the
Chebyshev series), a trace and a diagonal entry follow from the moments:
    tr f(X) = sum_m g_m tr T_m(X~) = N sum_m g_m d_m,
    f(X)_kk = sum_m g_m T_m(X~)_kk  (LDOS moments, Eq. (10); Eq. (12) estimates them).
Functions: "exp", f(lambda) = exp(p lambda) (Estrada index tr exp(A) at
p = 1, subgraph centrality exp(A)_kk, heat kernel exp(-t L) at p = -t) and
"resolvent", f(lambda) = 1 / (1 - p lambda) (resolvent centrality
((I - p A)^{-1})_kk), which needs 1 - p lambda != 0 on [a, b].  Nodes
without edges have eigenvalue 0 in A and L; each adds f(0) = 1 to a trace.

Readings (the paper names the quantities only): the coefficients g_m are
the Chebyshev interpolation coefficients of f on [a, b] at K = max(4M, 256)
Chebyshev-Gauss points (g_m = (2 - [m = 0]) / K sum_j f(c + r cos t_j)
cos(m t_j), t_j = pi (j + 1/2) / K); no damping kernel (f is smooth on the
interval, its coefficients decay geometrically).
"""
from __future__ import annotations

import numpy as np

from .kpm import Csr
from .operators import operator_matrix

__all__ = ["fn_values", "cheb_coeffs", "trace_fn", "diag_fn", "ldos_operator", "exact_fn_trace", "exact_fn_diag"]


def fn_values(fn: str, p: float, lam) -> np.ndarray:
    """f(lambda) for fn "exp" (exp(p lambda)) or "resolvent" (1 / (1 - p lambda))."""
    lam = np.asarray(lam, np.float64)
    if fn == "exp":
        return np.exp(p * lam)
    if fn == "resolvent":
        return 1.0 / (1.0 - p * lam)
    raise ValueError(fn)


def cheb_coeffs(fn: str, p: float, interval, m_count: int) -> np.ndarray:
    """g_0..g_{M-1} with f(c + r x) ~ sum_m g_m T_m(x) on [-1, 1]."""
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    k = max(4 * m_count, 256)
    t = np.pi * (np.arange(k) + 0.5) / k
    f = fn_values(fn, p, c + r * np.cos(t))
    g = np.array([(2.0 / k) * np.sum(f * np.cos(m * t)) for m in range(m_count)])
    g[0] *= 0.5
    return g


def trace_fn(d, g, n: int, n_isolated: int = 0) -> float:
    """tr f(X) = N sum_m g_m d_m over the nodes with edges, plus f(0) = 1 per
    node without edges (eigenvalue 0 of A and L)."""
    return float(n * np.dot(np.asarray(g), np.asarray(d)) + n_isolated)


def diag_fn(c_moments, g) -> np.ndarray:
    """f(X)_kk = sum_m g_m C[k, m] from LDOS moments C (N x M)."""
    return np.asarray(c_moments, np.float64) @ np.asarray(g, np.float64)


def ldos_operator(g: Csr, z: np.ndarray, m_count: int, op: str, interval):
    """Stochastic LDOS of X~ = (X - c) / r (Eq. (12) on X~): V_0 = Z,
    V_1 = X~ Z, V_{m+1} = 2 X~ V_m - V_{m-1};
    C[k, m] = (1/Nz) sum_j z_kj (V_m)_kj and d_m = sum_k C[k, m] / N.
    Returns (d (M,), C (N, M))."""
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    x = operator_matrix(g, op)
    z = np.asarray(z, np.float64)
    nz = z.shape[1]

    def apply(v):
        return (x @ v - c * v) / r

    cm = np.zeros((g.n, m_count))
    v_prev, v = z, apply(z)
    cm[:, 0] = np.sum(z * z, axis=1) / nz
    if m_count > 1:
        cm[:, 1] = np.sum(z * v, axis=1) / nz
    for m in range(2, m_count):
        v_prev, v = v, 2.0 * apply(v) - v_prev
        cm[:, m] = np.sum(z * v, axis=1) / nz
    return cm.sum(axis=0) / g.n, cm


def exact_fn_trace(g: Csr, op: str, fn: str, p: float, n_isolated: int = 0) -> float:
    """tr f(X) from the dense spectrum of X (plus f(0) per node without edges)."""
    lam = np.linalg.eigvalsh(operator_matrix(g, op).toarray())
    return float(np.sum(fn_values(fn, p, lam)) + n_isolated)


def exact_fn_diag(g: Csr, op: str, fn: str, p: float) -> np.ndarray:
    """f(X)_kk = sum_i q_i(k)^2 f(lambda_i) from the dense eigendecomposition."""
    lam, q = np.linalg.eigh(operator_matrix(g, op).toarray())
    return (q * q) @ fn_values(fn, p, lam)
