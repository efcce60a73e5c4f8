"""FP64 oracle of KPM on other graph operators (§2.1 operators, Eq. (5)).

TEST INFRASTRUCTURE ONLY (see the package header).

The adjacency A and the combinatorial Laplacian L = D - A have spectra outside
[-1, 1]; Eq. (5) maps an interval [a, b] holding the spectrum onto [-1, 1]
with X~ = (X - c) / r, c = (a + b) / 2, r = (b - a) / 2, and the Chebyshev
moments are those of X~.  Default interval (Gershgorin): [-d_max, d_max] for
A, [0, 2 d_max] for L.  The normalised Laplacian I - H and the random-walk
matrix D^{-1} A need no new recurrence: I - H - 1 = -H, so its moments are
(-1)^m d_m(H), and D^{-1} A = D^{-1/2} H D^{1/2} has the spectrum of H.

A tighter interval than Gershgorin's comes from the Lanczos process of §3.2
run on X itself: the extreme Ritz values theta of a probe's tridiagonal lie
inside the spectrum and move out toward its ends as steps are added; the
residual of a Ritz pair (theta, y = Z s) is ||X y - theta y|| = beta_M |s_M|
(s_M the last component of the tridiagonal's unit eigenvector), and beta_M
bounds it.  Reading (the paper gives no interval estimate): [min theta - r,
max theta + r] over the probes with r = beta_M ("residual": on 4 or more
probes it contained the spectrum of every graph tried, even after 3 steps) or
r = beta_M |s_M|
("ritz": the Ritz pair's own residual, tight once the extreme Ritz values
have converged, after ~30 steps on 4 or more probes, but too narrow before),
widened by pad (b - a) at each end, ends known exactly (lambda_max(H) = 1,
lambda_min(D - A) = 0, lambda_min(I - H) = 0) taken exactly, clipped to the
Gershgorin interval.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import eigh_tridiagonal

from .gql import lanczos
from .kpm import (Csr, cheb_values, closed_twin_classes, h_sparse, motif_classes, parallel_path_classes,
                  pendant_twin_classes, twin_classes)

__all__ = ["operator_matrix", "gershgorin_interval", "exact_operator_moments", "kpm_operator",
           "ritz_bounds", "spectral_interval", "motif_spikes"]


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


def ritz_bounds(alpha, beta, steps, bound: str = "residual") -> np.ndarray:
    """Per probe [theta_min - r, theta_max + r] (an (Nz, 2) array) from its
    Lanczos coefficients: theta the extreme eigenvalues of its tridiagonal,
    r = beta_M ("residual") or beta_M |s_M| ("ritz", s the unit eigenvector of
    that theta)."""
    out = np.zeros((alpha.shape[0], 2))
    for j in range(alpha.shape[0]):
        k = int(steps[j])
        if k > 1:
            theta, s = eigh_tridiagonal(alpha[j, :k], beta[j, :k - 1])
        else:
            theta, s = alpha[j, :1], np.ones((1, 1))
        r_lo = r_hi = abs(beta[j, k - 1])
        if bound == "ritz":
            r_lo, r_hi = r_lo * abs(s[-1, 0]), r_hi * abs(s[-1, -1])
        out[j] = theta[0] - r_lo, theta[-1] + r_hi
    return out


def spectral_interval(g: Csr, op: str, z: np.ndarray, m_steps: int, pad: float = 0.01, bound: str = "residual"):
    """[a, b] holding the spectrum of X ("adjacency", "laplacian",
    "normalized_adjacency", "normalized_laplacian") from m_steps Lanczos steps
    per probe column of z; bound "residual" or "ritz" (the reading in the
    module header)."""
    if op in ("adjacency", "laplacian"):
        x, (g_lo, g_hi) = operator_matrix(g, op), gershgorin_interval(g, op)
    else:
        x, (g_lo, g_hi) = h_sparse(g), ((-1.0, 1.0) if op == "normalized_adjacency" else (0.0, 2.0))
    alpha, beta, steps = lanczos(g, z, m_steps, x=x)
    per_probe = ritz_bounds(alpha, beta, steps, bound)
    lo, hi = per_probe[:, 0].min(), per_probe[:, 1].max()
    if op == "normalized_laplacian":  # Lanczos ran on H; the spectrum of I - H is 1 - that of H
        lo, hi = 1.0 - hi, 1.0 - lo
    w = hi - lo
    lo, hi = lo - pad * w, hi + pad * w
    if op in ("laplacian", "normalized_laplacian"):
        lo = 0.0
    if op == "normalized_adjacency":
        hi = 1.0
    return max(lo, g_lo), min(hi, g_hi)


def motif_spikes(g: Csr, op: str, open_twins: bool = True, closed_twins: bool = True, pendant_twins: bool = False,
                 parallel_paths: bool = False):
    """Eigenvalues of X that the motif classes of ``motif_classes`` take out
    (§3.4's motifs on §2.1's operators), as sorted (lambda, count) pairs.

    Members of a class share their degree, so the within-class difference
    vectors span the same invariant subspace of H, A and D - A; only the
    eigenvalue differs.  For a class of c members of degree d (c - 1
    eigenvalues each, two per pair for the two-class motifs):
      open twins        H 0             A 0     D - A  d
      closed twins      H -1/d          A -1    D - A  d + 1
      pendant twins     H +-1/sqrt(d)   A +-1   D - A  ((d + 1) +- sqrt((d - 1)^2 + 4)) / 2
      parallel paths    H +-1/2         A +-1   D - A  1, 3
    (on a node / leaf pair the operators act as [[0, 1], [1, 0]] (A) and
    [[d, -1], [-1, 1]] (D - A); on a path pair a - b as [[0, 1], [1, 0]] and
    [[2, -1], [-1, 2]]).  op "normalized_adjacency" gives motif_classes' own
    spikes, "normalized_laplacian" 1 - those."""
    if op in ("normalized_adjacency", "normalized_laplacian"):
        _, _, sp = motif_classes(g, open_twins, closed_twins, pendant_twins, parallel_paths)
        if op == "normalized_laplacian":
            sp = sorted((1.0 - x, c) for x, c in sp)
        return sp
    if op not in ("adjacency", "laplacian"):
        raise ValueError(op)
    lap = op == "laplacian"
    deg = np.diff(g.row_ptr)
    out: dict[float, int] = {}

    def add(x, c):
        out[float(x)] = out.get(float(x), 0) + int(c)

    if open_twins:
        oc, _ = twin_classes(g)
        for i in np.nonzero(oc != np.arange(g.n))[0]:
            add(float(deg[i]) if lap else 0.0, 1)
    if closed_twins:
        _, _, per_d = closed_twin_classes(g)
        for d, c in per_d.items():
            add(d + 1.0 if lap else -1.0, c)
    if pendant_twins:
        _, _, pairs = pendant_twin_classes(g)
        for d, c in pairs.items():
            if lap:
                r = np.sqrt((d - 1.0) ** 2 + 4.0)
                add((d + 1.0 - r) / 2.0, c)
                add((d + 1.0 + r) / 2.0, c)
            else:
                add(-1.0, c)
                add(1.0, c)
    if parallel_paths:
        _, _, pairs = parallel_path_classes(g)
        if pairs:
            add(1.0 if lap else -1.0, pairs)
            add(3.0 if lap else 1.0, pairs)
    return sorted(out.items())
