"""FP64 oracle of the kernel polynomial method for network DOS / LDOS.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Paper: Dong, Benson, Bindel, "Network Density of States", KDD 2019.
Section / equation references are to that paper; equation numbers follow the
order of the numbered displays: (1) DOS, (2) LDOS, (6) Chebyshev three-term
recurrence, (7) orthogonality weight, (8)-(9) DOS expansion and coefficients,
(10) PDOS coefficients, (11) trace estimator, (12) diagonal estimator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

__all__ = [
    "SPLITMIX64_GAMMA",
    "splitmix64",
    "probes",
    "Csr",
    "build_csr",
    "h_sparse",
    "dense_h",
    "exact_eigs",
    "cheb_values",
    "exact_moments",
    "exact_ldos",
    "kpm_direct",
    "kpm_doubled",
    "twin_classes",
    "closed_twin_classes",
    "motif_classes",
    "pendant_twin_classes",
    "parallel_path_classes",
    "project_probes",
    "jackson",
    "bin_edges",
    "bin_integrals",
    "histogram",
    "point_mass_histogram",
    "exact_histogram",
    "l1",
]

# ---------------------------------------------------------------------------
# Probe generator
# ---------------------------------------------------------------------------
# The paper's probes are i.i.d. with mean 0 and variance 1 (§3.1, before
# Eq. (11)); Rademacher (+-1) probes are used here.  The random bits come from
# SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): the n-th output (n = 0, 1, ...) of the stream
# seeded with s is mix(s + (n + 1) * GAMMA), where mix is the 64-bit
# variant-13 finalizer with the constants below.
#
# Probe definition: entry (i, j) of the probe block, for the node whose
# ORIGINAL id is o, uses counter n = ((j >> 6) << 32) | o, and
#     z[i, j] = +1 if bit (j & 63) of splitmix64(seed, n) is 0, else -1.
# Keying by the original id makes the probes independent of the node
# compaction and of any internal node order.

SPLITMIX64_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n) -> np.ndarray:
    """n-th SplitMix64 output(s) of the stream seeded with ``seed`` (uint64 array)."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (n + np.uint64(1)) * SPLITMIX64_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def probes(seed: int, old_id, nz: int) -> np.ndarray:
    """Rademacher probe block Z (N x nz, float64) for nodes with original ids ``old_id``."""
    old_id = np.asarray(old_id, dtype=np.uint64)
    z = np.empty((old_id.size, nz), np.float64)
    for j in range(nz):
        ctr = (np.uint64(j >> 6) << np.uint64(32)) | old_id
        bit = (splitmix64(seed, ctr) >> np.uint64(j & 63)) & np.uint64(1)
        z[:, j] = 1.0 - 2.0 * bit.astype(np.float64)
    return z


# ---------------------------------------------------------------------------
# Graph operator: normalized adjacency H = D^{-1/2} A D^{-1/2}  (§2.1)
# ---------------------------------------------------------------------------

@dataclass
class Csr:
    """CSR of the unweighted adjacency A after symmetrization and compaction.

    row_ptr int64[N+1], col int32[nnz] (ascending within a row), deg int32[N],
    s64 = 1/sqrt(deg) (float64), s32 = float32(s64), old_id int32[N] (original
    id of each kept node, ascending), n_isolated = original nodes dropped
    because they have no edge.
    """

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    deg: np.ndarray
    s64: np.ndarray
    s32: np.ndarray
    old_id: np.ndarray
    n_isolated: int
    n_original: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def build_csr(src, dst, n_nodes: int) -> Csr:
    """Undirected simple graph -> CSR of A, degrees and D^{-1/2}.

    §2.1 defines A for undirected graphs with a_ij > 0 on edges.  The workloads
    are unweighted, so repeated pairs collapse to one edge of weight 1 and
    self-loops (u == v) are removed.  Nodes of degree 0 make D^{-1/2}
    undefined; they contribute the eigenvalue 0 (§5.4 notes isolated nodes give
    lambda = 0), so they are compacted out of the operator, keeping the order of
    the original ids, and counted in ``n_isolated``.
    """
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    n_nodes = int(n_nodes)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n_nodes or dst.max() >= n_nodes):
        raise ValueError("edge endpoint out of range")
    keep = src != dst
    u = np.concatenate([src[keep], dst[keep]])
    v = np.concatenate([dst[keep], src[keep]])
    key = np.unique(u * np.int64(n_nodes) + v)  # sorted by (u, v), duplicates removed
    u = key // n_nodes
    v = key % n_nodes
    deg_full = np.bincount(u, minlength=n_nodes).astype(np.int64)
    old_id = np.nonzero(deg_full > 0)[0]
    new_id = np.full(n_nodes, -1, dtype=np.int64)
    new_id[old_id] = np.arange(old_id.size)
    deg = deg_full[old_id]
    row_ptr = np.zeros(old_id.size + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = new_id[v]
    s64 = 1.0 / np.sqrt(deg.astype(np.float64))
    return Csr(
        n=int(old_id.size),
        row_ptr=row_ptr,
        col=col.astype(np.int32),
        deg=deg.astype(np.int32),
        s64=s64,
        s32=s64.astype(np.float32),
        old_id=old_id.astype(np.int32),
        n_isolated=int(n_nodes - old_id.size),
        n_original=n_nodes,
    )


def h_sparse(g: Csr) -> sp.csr_matrix:
    """H = D^{-1/2} A D^{-1/2} as a scipy CSR matrix, H_ij = s_i s_j (§2.1)."""
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    vals = g.s64[rows] * g.s64[g.col]
    return sp.csr_matrix((vals, g.col.astype(np.int64), g.row_ptr), shape=(g.n, g.n))


def dense_h(g: Csr) -> np.ndarray:
    """Dense H (small graphs only)."""
    return h_sparse(g).toarray()


def exact_eigs(g: Csr):
    """Eigen-decomposition H = Q Lambda Q^T (§2.2), ascending eigenvalues."""
    lam, q = np.linalg.eigh(dense_h(g))
    return lam, q


def cheb_values(x, m_count: int) -> np.ndarray:
    """T_m(x) for m = 0..m_count-1 by the three-term recurrence, Eq. (6). Shape (m_count, len(x))."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((m_count,) + x.shape, np.float64)
    if m_count > 0:
        out[0] = 1.0
    if m_count > 1:
        out[1] = x
    for m in range(1, m_count - 1):
        out[m + 1] = 2.0 * x * out[m] - out[m - 1]
    return out


def exact_moments(lam, m_count: int) -> np.ndarray:
    """d_m = (1/N) sum_i T_m(lambda_i), Eq. (9)."""
    return cheb_values(lam, m_count).mean(axis=1)


def exact_ldos(lam, q, m_count: int) -> np.ndarray:
    """d_mk = sum_i q_i(k)^2 T_m(lambda_i) = T_m(H)_kk, Eq. (10).  Shape (N, m_count)."""
    t = cheb_values(lam, m_count)  # (M, N_eig)
    return (q * q) @ t.T


# ---------------------------------------------------------------------------
# Stochastic KPM (§3.1)
# ---------------------------------------------------------------------------

def kpm_direct(g: Csr, z: np.ndarray, m_count: int, ldos: bool = False):
    """Direct KPM moments with probe block Z (N x Nz).

    V_0 = Z, V_1 = H Z, V_{m+1} = 2 H V_m - V_{m-1}   (Eq. (6) applied to H).
    mu_m = sum_j z_j^T V_m e_j (trace estimator, Eq. (11), summed over probes).
    If ``ldos``: C[k, m] = (1/Nz) sum_j z_kj (V_m)_kj (diagonal estimator, Eq. (12)).
    Returns mu (m_count,) and C (N x m_count) or None.
    The normalised moments are d_m = mu_m / (N Nz).
    """
    h = h_sparse(g)
    z = np.asarray(z, dtype=np.float64)
    nz = z.shape[1]
    mu = np.zeros(m_count)
    c = np.zeros((g.n, m_count)) if ldos else None
    v_prev, v = None, z.copy()
    for m in range(m_count):
        if m == 1:
            v_prev, v = v, h @ v
        elif m >= 2:
            v_prev, v = v, 2.0 * (h @ v) - v_prev
        zv = z * v
        mu[m] = zv.sum()
        if ldos:
            c[:, m] = zv.sum(axis=1) / nz
    return mu, c


def kpm_doubled(g: Csr, z: np.ndarray, m_count: int) -> np.ndarray:
    """KPM moments from floor(M/2) matrix products using the doubling identities.

    Per probe, T_{2k} = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1
    (products of Chebyshev polynomials, from Eq. (6)), so with V_k = T_k(H) Z:
        mu_{2k}   = 2 <V_k, V_k>     - <V_0, V_0>
        mu_{2k+1} = 2 <V_{k+1}, V_k> - <V_1, V_0>
    where <X, Y> = sum of elementwise products.  Equal to ``kpm_direct`` up to
    rounding.  The moments are taken as V_k is formed, so only V_{k-1} and V_k
    are held (the 1.1M-node workload at M = 500 would otherwise hold 251
    blocks).
    """
    h = h_sparse(g)
    z = np.asarray(z, dtype=np.float64)
    k_max = m_count // 2
    mu = np.zeros(m_count)
    mu0 = np.sum(z * z)
    mu[0] = mu0
    if m_count < 2:
        return mu
    v_prev, v = z, h @ z  # V_0, V_1
    mu1 = np.sum(v * v_prev)
    mu[1] = mu1
    for k in range(1, k_max + 1):
        # here v = V_k and v_prev = V_{k-1}
        if 2 * k < m_count:
            mu[2 * k] = 2.0 * np.sum(v * v) - mu0
        if k >= 2 and 2 * k - 1 < m_count:
            mu[2 * k - 1] = 2.0 * np.sum(v * v_prev) - mu1
        if k < k_max:
            v_prev, v = v, 2.0 * (h @ v) - v_prev
    return mu


# ---------------------------------------------------------------------------
# Motif filtering, twin (lambda = 0) motif  (§3.4)
# ---------------------------------------------------------------------------

def twin_classes(g: Csr):
    """Classes of nodes with identical (open) neighbourhoods.

    Two dangling nodes on the same neighbour (Fig. 3a) -- and more generally any
    nodes i != j with N(i) = N(j) -- give eigenvectors e_i - e_j of H with
    eigenvalue 0 (§3.4).  The paper finds such pairs by hashing w = Hz and
    matching equal w_i "with high probability"; the oracle uses the exact
    relation the hash detects: equal sorted neighbour lists.
    Returns class_id int32[N] (the smallest member id of each class) and the
    number of removed eigenvalues sum_classes (c - 1).
    """
    class_id = np.arange(g.n, dtype=np.int32)
    first: dict[bytes, int] = {}
    rp, col = g.row_ptr, g.col
    for i in range(g.n):
        key = col[rp[i]:rp[i + 1]].tobytes()
        class_id[i] = first.setdefault(key, i)
    removed = int(g.n - len(first))
    return class_id, removed


def closed_twin_classes(g: Csr):
    """Classes of nodes with identical closed neighbourhoods N[i] = N(i) + {i}.

    Such nodes i != j are adjacent (j is in N[i]) and share the degree d; for
    them H (e_i - e_j) = -(e_i - e_j) / d (A (e_i - e_j) = e_j - e_i), so each
    class of size c carries c - 1 eigenvalues -1/d on localized eigenvectors
    (the lambda = -1/d motifs of §3.4, Fig. 3; d = 2: the triangle with two
    degree-2 nodes, lambda = -1/2).  Exact relation: equal sorted closed
    neighbour lists.
    Returns class_id int32[N] (smallest member), the removed count
    sum (c - 1), and {d: number of eigenvalues at -1/d}.
    """
    class_id = np.arange(g.n, dtype=np.int32)
    first: dict[bytes, int] = {}
    rp, col = g.row_ptr, g.col
    for i in range(g.n):
        nb = col[rp[i]:rp[i + 1]]
        key = np.sort(np.append(nb, np.int32(i))).astype(np.int32).tobytes()
        class_id[i] = first.setdefault(key, i)
    removed = int(g.n - len(first))
    spikes: dict[int, int] = {}
    for i in np.nonzero(class_id != np.arange(g.n))[0]:
        d = int(rp[i + 1] - rp[i])
        spikes[d] = spikes.get(d, 0) + 1
    return class_id, removed, spikes


def pendant_twin_classes(g: Csr):
    """Classes of pendant twins (§3.4, Fig. 3: the +-1/sqrt 2 and +-1/2 motifs).

    A node a of degree d >= 2 with exactly one leaf neighbour a' (d(a') = 1) is
    eligible; eligible a, b are pendant twins if N(a) - {a'} = N(b) - {b'} (so
    d(a) = d(b) = d and a, b are not adjacent).  For a class of c such nodes
    the vectors that sum to zero over the nodes and over their leaves form an
    invariant subspace of H on which H acts as [[0, 1/sqrt d], [1/sqrt d, 0]]
    per pair (H_{a a'} = 1/sqrt(d), the common neighbours cancel): c - 1
    eigenvalues at each of +-1/sqrt(d).  d = 2 is the pendant 2-path
    u - a - a' (+-1/sqrt 2), d = 4 the +-1/2 motif with three common
    neighbours.  The nodes form one class and their leaves another.
    Returns class_id (smallest member), the removed count 2 sum (c - 1), and
    {d: number of removed pairs}.
    """
    class_id = np.arange(g.n, dtype=np.int32)
    rp, col = g.row_ptr, g.col
    deg = np.diff(rp)
    groups: dict[bytes, list] = {}
    for a in range(g.n):
        if deg[a] < 2:
            continue
        nb = col[rp[a]:rp[a + 1]]
        leaves = nb[deg[nb] == 1]
        if leaves.size != 1:
            continue
        rest = nb[nb != leaves[0]]
        groups.setdefault(rest.astype(np.int32).tobytes(), []).append((a, int(leaves[0])))
    pairs: dict[int, int] = {}
    for lst in groups.values():
        if len(lst) < 2:
            continue
        f1 = min(a for a, _ in lst)
        f2 = min(x for _, x in lst)
        for a, x in lst:
            class_id[a] = f1
            class_id[x] = f2
        d = int(deg[lst[0][0]])
        pairs[d] = pairs.get(d, 0) + len(lst) - 1
    return class_id, 2 * sum(pairs.values()), pairs


def parallel_path_classes(g: Csr):
    """Classes of parallel 2-node paths between two hosts (the first +-1/2
    drawing of §3.4, Fig. 3).

    A path E - a - b - F with d(a) = d(b) = 2 and hosts E != F of degree >= 3
    (E = F would make a, b closed twins; a degree-2 host is itself a path node
    and would let instances overlap, as on a cycle, so such instances are
    left unfiltered).  If c >= 2 such paths join the same hosts, the
    nodes next to the smaller host form one class and those next to the
    larger host another; the vectors summing to zero over each carry c - 1
    eigenvalues at each of +-1/2 (H_ab = 1/2, the hosts see zero sums).
    Returns class_id (smallest member), the removed count 2 sum (c - 1) and
    the number of removed pairs.
    """
    class_id = np.arange(g.n, dtype=np.int32)
    rp, col = g.row_ptr, g.col
    deg = np.diff(rp)
    groups: dict[tuple, list] = {}
    for a in range(g.n):
        if deg[a] != 2:
            continue
        for b in col[rp[a]:rp[a + 1]]:
            b = int(b)
            if b <= a or deg[b] != 2:
                continue
            na, nb = col[rp[a]:rp[a + 1]], col[rp[b]:rp[b + 1]]
            e = int(na[0] if na[1] == b else na[1])
            f = int(nb[0] if nb[1] == a else nb[1])
            if e == f or deg[e] < 3 or deg[f] < 3:
                continue
            first, second = (a, b) if e < f else (b, a)
            groups.setdefault((min(e, f), max(e, f)), []).append((first, second))
    pairs = 0
    for lst in groups.values():
        if len(lst) < 2:
            continue
        f1 = min(x for x, _ in lst)
        f2 = min(y for _, y in lst)
        for x, y in lst:
            class_id[x] = f1
            class_id[y] = f2
        pairs += len(lst) - 1
    return class_id, 2 * pairs, pairs


def motif_classes(g: Csr, open_twins: bool = True, closed_twins: bool = True, pendant_twins: bool = False,
                  parallel_paths: bool = False):
    """Open-twin, closed-twin and (optionally) pendant-twin classes together (§3.4).

    The relations are disjoint: if N(i) = N(j) and N[i] = N[k] (k != i), then k
    is in N(i) = N(j), so j ~ k, while j would have to lie in N[k] = N[i],
    which holds neither j (not adjacent to i) nor i's other members.  So every
    node is in at most one nontrivial class and one class-mean projection
    filters both kinds.  Returns class_id, the removed count and the removed
    eigenvalues as a list of (lambda, count) sorted by lambda.
    """
    ident = np.arange(g.n, dtype=np.int32)
    cid = ident.copy()
    removed = 0
    spikes = []
    in_open = np.zeros(g.n, bool)
    if open_twins:
        oc, r0 = twin_classes(g)
        in_open = np.bincount(oc, minlength=g.n)[oc] >= 2
        cid = np.where(in_open, oc, cid)
        removed += r0
        if r0:
            spikes.append((0.0, r0))
    taken = in_open.copy()
    if closed_twins:
        cc, r1, sp = closed_twin_classes(g)
        in_closed = np.bincount(cc, minlength=g.n)[cc] >= 2
        assert not np.any(taken & in_closed)
        taken |= in_closed
        cid = np.where(in_closed, cc, cid)
        removed += r1
        spikes.extend((-1.0 / d, c) for d, c in sp.items())
    if pendant_twins:
        pc, r2, pairs = pendant_twin_classes(g)
        in_pt = np.bincount(pc, minlength=g.n)[pc] >= 2
        assert not np.any(taken & in_pt)
        cid = np.where(in_pt, pc, cid)
        removed += r2
        for d, c in pairs.items():
            r = 1.0 / np.sqrt(float(d))
            spikes.extend([(-r, c), (r, c)])
        taken |= in_pt
    if parallel_paths:
        qc, r3, pairs = parallel_path_classes(g)
        in_pp = np.bincount(qc, minlength=g.n)[qc] >= 2
        assert not np.any(taken & in_pp)
        cid = np.where(in_pp, qc, cid)
        removed += r3
        if pairs:
            spikes.extend([(-0.5, pairs), (0.5, pairs)])
    # equal eigenvalues from different motifs (e.g. -1/2) are one spike
    merged: dict[float, int] = {}
    for x, c in spikes:
        merged[x] = merged.get(x, 0) + c
    return cid, removed, sorted(merged.items())


def project_probes(z: np.ndarray, class_id: np.ndarray) -> np.ndarray:
    """Z_r = P P^T Z: each class's rows replaced by their mean (§3.4).

    P has one orthonormal column per class (the normalised class indicator), so
    P P^T averages over each class.
    """
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[0]
    sums = np.zeros_like(z)
    np.add.at(sums, class_id, z)
    cnt = np.bincount(class_id, minlength=n).astype(np.float64)
    return sums[class_id] / cnt[class_id][:, None]


# ---------------------------------------------------------------------------
# Density reconstruction: Jackson damping and spectral histogram
# ---------------------------------------------------------------------------

def jackson(m_count: int) -> np.ndarray:
    """Jackson damping factors g_m for a series with m_count terms (m = 0..M-1).

    §3.1 and Jackson's theorem (§4.1) name the factors but do not print them;
    this is the Jackson kernel of the KPM review the paper cites for KPM
    (Weisse et al. 2006, with that review's N = m_count):
    g_m = [(M - m + 1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))] / (M+1).
    """
    m = np.arange(m_count, dtype=np.float64)
    a = np.pi / (m_count + 1)
    return ((m_count - m + 1) * np.cos(a * m) + np.sin(a * m) / np.tan(a)) / (m_count + 1)


def bin_edges(n_bins: int) -> np.ndarray:
    """Equal-width bins over [-1, 1] (the spectral histogram of §2.2)."""
    return np.linspace(-1.0, 1.0, n_bins + 1)


def bin_integrals(m_count: int, n_bins: int) -> np.ndarray:
    """I[m, b] = integral over bin b of T_m(x) / (pi sqrt(1 - x^2)) dx.

    With x = cos(theta): I[0, b] = (theta_a - theta_b)/pi and, for m >= 1,
    I[m, b] = (sin(m theta_a) - sin(m theta_b)) / (m pi), theta = arccos(edge).
    """
    e = bin_edges(n_bins)
    th = np.arccos(np.clip(e, -1.0, 1.0))
    ta, tb = th[:-1], th[1:]
    out = np.empty((m_count, n_bins))
    out[0] = (ta - tb) / np.pi
    for m in range(1, m_count):
        out[m] = (np.sin(m * ta) - np.sin(m * tb)) / (m * np.pi)
    return out


def histogram(d, n_bins: int, kernel: str = "jackson") -> np.ndarray:
    """Bin masses of the truncated (damped) DOS expansion.

    mu(x) = [g_0 d_0 + 2 sum_{m>=1} g_m d_m T_m(x)] / (pi sqrt(1 - x^2)):
    Eq. (8) with the weight of Eq. (7), reading the sum in Eq. (8) as starting
    at m = 0 and delta_{0n} in Eq. (7) as delta_{0m}; g_m = 1 without damping.
    Bin b's mass is g_0 d_0 I[0,b] + 2 sum_{m>=1} g_m d_m I[m,b].
    """
    d = np.asarray(d, dtype=np.float64)
    m_count = d.size
    g = jackson(m_count) if kernel == "jackson" else np.ones(m_count)
    coef = 2.0 * g * d
    coef[0] = g[0] * d[0]
    return coef @ bin_integrals(m_count, n_bins)


def point_mass_histogram(points, weights, n_bins: int, tol: float = 1e-9) -> np.ndarray:
    """Histogram of point masses on [-1, 1].

    A point within ``tol`` of an interior edge splits its weight evenly between
    the two bins; points at +-1 go to the end bins.
    """
    e = bin_edges(n_bins)
    h = np.zeros(n_bins)
    width = 2.0 / n_bins
    for x, w in zip(np.asarray(points, float).ravel(), np.asarray(weights, float).ravel()):
        x = min(max(x, -1.0), 1.0)
        k = int(round((x + 1.0) / width))
        if 0 < k < n_bins and abs(x - e[k]) <= tol:
            h[k - 1] += 0.5 * w
            h[k] += 0.5 * w
        else:
            b = int(np.floor((x + 1.0) / width))
            h[min(max(b, 0), n_bins - 1)] += w
    return h


def exact_histogram(lam, n_bins: int, n_total: int | None = None, n_extra_zero: int = 0) -> np.ndarray:
    """Spectral histogram of a known spectrum: eigenvalue counts per bin / N.

    ``n_extra_zero`` eigenvalues at 0 (isolated nodes) are added; N = n_total
    (default len(lam) + n_extra_zero).
    """
    lam = np.asarray(lam, float)
    n_total = lam.size + n_extra_zero if n_total is None else n_total
    pts = np.concatenate([lam, np.zeros(n_extra_zero)])
    return point_mass_histogram(pts, np.full(pts.size, 1.0 / n_total), n_bins)


def l1(h, h_ref) -> float:
    """L1 distance of two bin-mass vectors (the 'relative L1 error' of Fig. 4)."""
    return float(np.abs(np.asarray(h, float) - np.asarray(h_ref, float)).sum())
