"""FP64 oracle of KPM on other graph operators (§2.1 operators, Eq. (5)).

TEST INFRASTRUCTURE ONLY (see the package header).

The adjacency A and the combinatorial Laplacian L = D - A have spectra outside
[-1, 1]; Eq. (5) maps an interval [a, b] holding the spectrum onto [-1, 1]
with X~ = (X - c) / r, c = (a + b) / 2, r = (b - a) / 2, and the Chebyshev
moments are those of X~.  Default interval (Gershgorin): [-d_max, d_max] for
A, [0, 2 d_max] for L.  The normalised Laplacian I - H and the random-walk
matrix D^{-1} A need no new recurrence: I - H - 1 = -H, so its moments are
(-1)^m d_m(H), and D^{-1} A = D^{-1/2} H D^{1/2} has the spectrum of H.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .kpm import Csr, cheb_values

__all__ = ["operator_matrix", "gershgorin_interval", "exact_operator_moments", "kpm_operator"]


def operator_matrix(g: Csr, op: str) -> sp.csr_matrix:
    """A ("adjacency") or L = D - A ("laplacian") of the compacted graph."""
    a = sp.csr_matrix((np.ones(g.col.size), g.col.astype(np.int64), g.row_ptr), shape=(g.n, g.n))
    if op == "adjacency":
        return a
    if op == "laplacian":
        return (sp.diags(np.diff(g.row_ptr).astype(np.float64)) - a).tocsr()
    raise ValueError(op)


def gershgorin_interval(g: Csr, op: str):
    """[a, b] from Gershgorin discs: every eigenvalue lies in [-d_max, d_max]
    for A and in [0, 2 d_max] for L (row sums of |entries|)."""
    dmax = float(np.diff(g.row_ptr).max()) if g.n else 0.0
    return (-dmax, dmax) if op == "adjacency" else (0.0, 2.0 * dmax)


def exact_operator_moments(g: Csr, op: str, interval, m_count: int) -> np.ndarray:
    """d_m = (1/N) sum_i T_m((lambda_i - c) / r) from the dense spectrum."""
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    lam = np.linalg.eigvalsh(operator_matrix(g, op).toarray())
    return cheb_values((lam - c) / r, m_count).mean(axis=1)


def kpm_operator(g: Csr, z: np.ndarray, m_count: int, op: str, interval) -> np.ndarray:
    """Stochastic moments of X~ = (X - c) / r by the three-term recurrence
    (Eq. (6) on X~): V_0 = Z, V_1 = X~ Z, V_{m+1} = 2 X~ V_m - V_{m-1};
    d_m = sum_j z_j^T V_m e_j / (N Nz) (Eq. (11))."""
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    x = operator_matrix(g, op)
    z = np.asarray(z, np.float64)

    def apply(v):
        return (x @ v - c * v) / r

    mu = np.zeros(m_count)
    v_prev, v = z, apply(z)
    mu[0] = np.sum(z * z)
    if m_count > 1:
        mu[1] = np.sum(z * v)
    for m in range(2, m_count):
        v_prev, v = v, 2.0 * apply(v) - v_prev
        mu[m] = np.sum(z * v)
    return mu / (g.n * z.shape[1])
