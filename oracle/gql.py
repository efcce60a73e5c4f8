"""FP64 oracle of the Gauss quadrature / Lanczos (GQL) estimator (§3.2).

TEST INFRASTRUCTURE ONLY (see the package header).

For a probe z, M Lanczos steps on H give H Z_M = Z_M Gamma_M + r_M e_M^T with
Z_M orthonormal and Gamma_M = tridiag(beta; alpha; beta).  The Gauss rule of
the probe's spectral measure has the eigenvalues tau_i of Gamma_M as nodes
and the squared first eigenvector components |p_i1|^2 as weights:
    z^T f(H) z ~ ||z||^2 sum_i |p_i1|^2 f(tau_i),
exact for polynomials f of degree <= 2M - 1 (a Gauss rule with M nodes; the
paper prints 2M + 1, read here as the standard Gauss degree 2M - 1).
Averaged over Nz probes (||z||^2 = N for Rademacher probes), the rules
estimate the DOS; their Chebyshev moments estimate d_m.

Reading: plain Lanczos without reorthogonalisation (the paper names none);
a probe whose Krylov space is exhausted (beta_k <= 1e-10 ||z||) stops there
and keeps the k-node rule, which is then exact for every polynomial.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal

from .kpm import Csr, h_sparse, point_mass_histogram

__all__ = ["lanczos", "gauss_rules", "gql_moments", "gql_histogram"]


def lanczos(g: Csr, z: np.ndarray, m_steps: int, x=None):
    """Lanczos coefficients of each probe column (§3.2) on H, or on the
    symmetric sparse operator x of the same graph (A or D - A, §2.1).

    Returns alpha (Nz, M), beta (Nz, M) (beta[:, k] couples steps k and k+1;
    the last column is the residual norm) and steps (Nz,) = the number of
    steps each probe ran (M, or fewer after a breakdown)."""
    h = h_sparse(g) if x is None else x
    z = np.asarray(z, np.float64)
    nz = z.shape[1]
    alpha = np.zeros((nz, m_steps))
    beta = np.zeros((nz, m_steps))
    steps = np.zeros(nz, np.int64)
    for j in range(nz):
        norm0 = np.linalg.norm(z[:, j])
        v = z[:, j] / norm0
        v_prev = np.zeros_like(v)
        b_prev = 0.0
        for k in range(m_steps):
            w = h @ v
            a = float(v @ w)
            w = w - a * v - b_prev * v_prev
            b = float(np.linalg.norm(w))
            alpha[j, k] = a
            beta[j, k] = b
            steps[j] = k + 1
            if b <= 1e-10 * norm0:
                break
            v_prev, v, b_prev = v, w / b, b
    return alpha, beta, steps


def gauss_rules(alpha, beta, steps):
    """Per probe: nodes tau (eigenvalues of Gamma) and weights |p_1|^2."""
    rules = []
    for j in range(alpha.shape[0]):
        k = int(steps[j])
        tau, p = eigh_tridiagonal(alpha[j, :k], beta[j, :k - 1])
        rules.append((tau, p[0, :] ** 2))
    return rules


def gql_moments(alpha, beta, steps, m_count: int, norms2=None, n: int | None = None):
    """Chebyshev moments of the averaged rules: d_m = (1/Nz) sum_j (||z_j||^2 / N)
    sum_i w_ij T_m(tau_ij) (Rademacher probes: ||z||^2 = N, the factor is 1)."""
    rules = gauss_rules(alpha, beta, steps)
    nz = len(rules)
    scale = np.ones(nz) if norms2 is None else np.asarray(norms2, float) / n
    d = np.zeros(m_count)
    for (tau, w), s in zip(rules, scale):
        t = np.arccos(np.clip(tau, -1.0, 1.0))
        d += s * (w[None, :] * np.cos(np.arange(m_count)[:, None] * t[None, :])).sum(axis=1)
    return d / nz


def gql_histogram(alpha, beta, steps, n_bins: int, norms2=None, n: int | None = None):
    """Bin masses of the averaged rules' point masses (the GQL density)."""
    rules = gauss_rules(alpha, beta, steps)
    nz = len(rules)
    scale = np.ones(nz) if norms2 is None else np.asarray(norms2, float) / n
    pts = np.concatenate([tau for tau, _ in rules])
    wts = np.concatenate([s * w / nz for (_, w), s in zip(rules, scale)])
    return point_mass_histogram(pts, wts, n_bins)
