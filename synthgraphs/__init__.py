"""Seeded synthetic graph generators.

These produce the edge lists that both the CPU oracle and the CUDA library
consume.  They hold none of the density-of-states arithmetic: each function
returns plain ``(src, dst, n_nodes)`` int64 edge lists (undirected edges, one
entry per sampled pair; duplicates and self-loops may occur and are left for the
CSR builder to remove) and is deterministic for a given seed.

The graph models follow the ones the paper works with:

* Erdos-Renyi G(n, p) -- every unordered pair independently with probability p
  (random-graph background of §2.1).
* Chung-Lu expected-degree graphs with a power-law weight sequence, standing
  in for the heavy-tailed SNAP networks of §5 (Table 1 sizes).
* Barabasi-Albert preferential attachment with m edges per new node (§5.3,
  "Model Verification").
* Twin-leaf injection: pairs of degree-1 leaves hung on a common host, the
  lambda = 0 motif of §3.4 (Fig. 3a).

Recipes (the parameters of each model) are stated in each function's
docstring.  Randomness comes from ``numpy.random.Generator(PCG64(seed))``,
except for Barabasi-Albert, whose sequential attachment runs in a small C
helper (``_native.c``, built with gcc on first use) drawing from SplitMix64.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

__all__ = [
    "erdos_renyi",
    "chung_lu",
    "chung_lu_device",
    "chung_lu_device_member",
    "barabasi_albert",
    "add_twin_leaves",
    "add_triangle_twins",
    "add_pendant_twins",
    "add_parallel_paths",
    "cycle",
    "complete",
    "star",
    "windmill",
    "grid2d",
    "random_geometric",
    "spider",
    "complete_bipartite",
    "path",
    "batch_graphs",
    "chung_lu_twins_family",
    "chung_lu_twins_member",
    "union",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


_HERE = os.path.dirname(os.path.abspath(__file__))
_native = None


def _native_lib():
    """The C helpers (_native.c), built with gcc on first use."""
    global _native
    if _native is None:
        so = os.path.join(_HERE, "_native.so")
        src = os.path.join(_HERE, "_native.c")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.ba_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64] + [ctypes.c_void_p] * 3
        lib.ba_edges.restype = ctypes.c_int64
        _native = lib
    return _native


def _pair_from_linear(idx: np.ndarray, n: int):
    """Map linear indices of the strict upper triangle (row-major) to (u, v), u < v."""
    idx = idx.astype(np.int64)
    # row u starts at offset(u) = u*(2n-u-1)/2
    nn = 2 * n - 1
    u = np.floor((nn - np.sqrt(np.maximum(nn * nn - 8.0 * idx, 0.0))) / 2.0).astype(np.int64)
    u = np.clip(u, 0, n - 2)

    def off(x):
        return x * (2 * n - x - 1) // 2

    # fix floating point off-by-one in both directions
    for _ in range(3):
        too_big = off(u) > idx
        u = np.where(too_big, u - 1, u)
        too_small = off(u + 1) <= idx
        u = np.where(too_small, u + 1, u)
    v = idx - off(u) + u + 1
    return u, v


def erdos_renyi(n: int, p: float, seed: int):
    """G(n, p): each of the n(n-1)/2 unordered pairs is an edge with probability p.

    Sampled by geometric skipping over the row-major strict upper triangle, so
    the cost is proportional to the number of edges.  Returns unique pairs u < v.
    """
    n = int(n)
    total = n * (n - 1) // 2
    if n < 2 or p <= 0.0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), n
    rng = _rng(seed)
    expect = total * p
    chunk = int(expect + 6.0 * math.sqrt(expect + 1.0) + 16)
    pos = []
    last = -1
    while True:
        gaps = rng.geometric(p, size=chunk).astype(np.int64)
        cs = last + np.cumsum(gaps)
        keep = cs[cs < total]
        pos.append(keep)
        if keep.size < cs.size:
            break
        last = int(cs[-1])
    lin = np.concatenate(pos) if pos else np.zeros(0, np.int64)
    u, v = _pair_from_linear(lin, n)
    return u, v, n


def chung_lu(n: int, gamma: float, mean_degree: float, seed: int, i0: float = 10.0):
    """Chung-Lu style power-law graph (fast endpoint-sampling variant).

    Node weights w_i = (i + i0)^(-1/(gamma-1)), i = 0..n-1, scaled so their
    mean is ``mean_degree`` (so hubs have the low ids).  round(n*mean_degree/2)
    edges are drawn, each endpoint independently with probability proportional
    to w.  Self-loops and repeated pairs are kept in the list (the CSR builder
    removes them), so realised degrees are slightly below the weights; nodes
    with no edge stay isolated.
    """
    rng = _rng(seed)
    i = np.arange(n, dtype=np.float64)
    w = (i + i0) ** (-1.0 / (gamma - 1.0))
    w *= mean_degree * n / w.sum()
    m = int(round(n * mean_degree / 2.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    src = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    dst = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    np.minimum(src, n - 1, out=src)
    np.minimum(dst, n - 1, out=dst)
    return src, dst, n


def chung_lu_device(n: int, gamma: float, mean_degree: float, seed: int, device="cuda", i0: float = 10.0,
                    chunk: int = 1 << 27):
    """The Chung-Lu model of chung_lu, drawn with torch on a CUDA device for
    graphs too large to generate on the host (1e9 edges): the same weights and
    endpoint sampling (uniforms searched in the cumulative weights), from a
    seeded torch generator on the device, so the draws differ from
    chung_lu's.  Returns int64 device tensors src, dst and n."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    i = torch.arange(n, dtype=torch.float64, device=device)
    w = (i + i0) ** (-1.0 / (gamma - 1.0))
    w *= mean_degree * n / w.sum()
    m = int(round(n * mean_degree / 2.0))
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    del i, w
    src = torch.empty(m, dtype=torch.int64, device=device)
    dst = torch.empty(m, dtype=torch.int64, device=device)
    for out in (src, dst):
        for off in range(0, m, chunk):
            k = min(chunk, m - off)
            u = torch.rand(k, generator=gen, dtype=torch.float64, device=device)
            out[off:off + k] = torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)
            del u
    return src, dst, n


def chung_lu_device_member(seed: int, n_min: int = 10_000, n_max: int = 1_000_000, deg_min: float = 5.0,
                           deg_max: float = 40.0, device="cuda"):
    """One graph of the large Chung-Lu family, drawn on the device: N
    log-uniform in [n_min, n_max], exponent uniform in [2.1, 3.0], mean
    degree uniform in [deg_min, deg_max] (parameters from numpy PCG64(seed),
    edges from chung_lu_device)."""
    rng = _rng(seed)
    n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    gam = float(rng.uniform(2.1, 3.0))
    md = float(rng.uniform(deg_min, deg_max))
    return chung_lu_device(n, gam, md, int(rng.integers(0, 2**62)), device=device)


def barabasi_albert(n: int, m: int, seed: int):
    """Barabasi-Albert preferential attachment.

    Seed graph: the clique K_{m+1} on nodes 0..m.  Each later node t attaches to
    m distinct earlier nodes, each drawn with probability proportional to its
    current degree (uniform draws from the list of edge endpoints, redrawing
    repeats).  The draws use SplitMix64 seeded with ``seed`` (C helper).
    Returns unique pairs.
    """
    n, m = int(n), int(m)
    if n <= m + 1:
        return complete(n)
    if not 1 <= m <= 64:
        raise ValueError("m must be in [1, 64]")
    n_edges = m * (m + 1) // 2 + (n - m - 1) * m
    src = np.empty(n_edges, np.int64)
    dst = np.empty(n_edges, np.int64)
    ends = np.empty(2 * n_edges, np.int64)
    got = _native_lib().ba_edges(n, m, int(seed) & (2**64 - 1), src.ctypes.data, dst.ctypes.data, ends.ctypes.data)
    assert got == n_edges
    return src, dst, n


def watts_strogatz(n: int, k: int, p: float, seed: int):
    """Watts-Strogatz small world: the ring lattice joining each node to its k
    nearest neighbours on each side, then each lattice edge (i, i + j) has its
    far end moved, with probability p, to a uniformly drawn node that is
    neither i nor already a neighbour of i (numpy PCG64).  Returns unique pairs."""
    n, k = int(n), int(k)
    if not 1 <= k < n // 2:
        raise ValueError("need 1 <= k < n / 2")
    rng = _rng(seed)
    nbr = [set() for _ in range(n)]
    for i in range(n):
        for j in range(1, k + 1):
            nbr[i].add((i + j) % n)
            nbr[(i + j) % n].add(i)
    for j in range(1, k + 1):
        for i in range(n):
            v = (i + j) % n
            if v not in nbr[i] or rng.random() >= p:
                continue
            w = int(rng.integers(n))
            if w == i or w in nbr[i]:
                continue  # no move when the draw hits i or a neighbour
            nbr[i].discard(v)
            nbr[v].discard(i)
            nbr[i].add(w)
            nbr[w].add(i)
    src = np.array([i for i in range(n) for v in nbr[i] if i < v], np.int64)
    dst = np.array([v for i in range(n) for v in nbr[i] if i < v], np.int64)
    return src, dst, n


def add_twin_leaves(src, dst, n: int, n_hosts: int, seed: int):
    """Hang two new degree-1 leaves on each of ``n_hosts`` hosts.

    Hosts are drawn without replacement from the nodes that have at least one
    edge in (src, dst) that is not a self-loop.  The two leaves of host h get
    the ids n + 2k and n + 2k + 1 (k = the host's draw index).  Each pair is an
    instance of the lambda = 0 twin motif (§3.4, Fig. 3a).  Returns the
    extended edge list and the new node count n + 2*n_hosts.
    """
    rng = _rng(seed)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    live = np.zeros(n, bool)
    nl = src != dst
    live[src[nl]] = True
    live[dst[nl]] = True
    cand = np.nonzero(live)[0]
    hosts = rng.choice(cand, size=int(n_hosts), replace=False).astype(np.int64)
    leaves = n + np.arange(2 * n_hosts, dtype=np.int64)
    new_src = np.concatenate([src, np.repeat(hosts, 2)])
    new_dst = np.concatenate([dst, leaves])
    return new_src, new_dst, n + 2 * int(n_hosts)


def add_triangle_twins(src, dst, n: int, n_hosts: int, seed: int):
    """Hang a triangle on each of ``n_hosts`` hosts: two new nodes a, b joined
    to the host and to each other.  a and b then have equal closed
    neighbourhoods (the lambda = -1/2 motif of §3.4, Fig. 3).  Hosts are drawn
    without replacement among the nodes with a non-loop edge; host k's new
    nodes get ids n + 2k and n + 2k + 1.  Returns the extended edge list and
    n + 2 * n_hosts.
    """
    rng = _rng(seed)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    live = np.zeros(n, bool)
    nl = src != dst
    live[src[nl]] = True
    live[dst[nl]] = True
    hosts = rng.choice(np.nonzero(live)[0], size=int(n_hosts), replace=False).astype(np.int64)
    a = n + 2 * np.arange(n_hosts, dtype=np.int64)
    b = a + 1
    new_src = np.concatenate([src, hosts, hosts, a])
    new_dst = np.concatenate([dst, a, b, b])
    return new_src, new_dst, n + 2 * int(n_hosts)


def spider(legs: int, length: int = 2):
    """Spider: centre 0 with `legs` paths of `length` nodes each; legs of
    length 2 are pendant 2-paths sharing the host 0 (the +-1/sqrt(2) motif)."""
    src, dst = [], []
    nxt = 1
    for _ in range(legs):
        prev = 0
        for _ in range(length):
            src.append(prev)
            dst.append(nxt)
            prev = nxt
            nxt += 1
    return np.asarray(src, np.int64), np.asarray(dst, np.int64), nxt


def add_pendant_twins(src, dst, n: int, n_groups: int, k_common: int, seed: int):
    """Add ``n_groups`` pairs of pendant twins: two new nodes a, b joined to the
    same ``k_common`` existing nodes (drawn without replacement among the
    nodes with a non-loop edge) and each to a new leaf of its own, so
    N(a) - {a'} = N(b) - {b'} and d(a) = d(b) = k_common + 1 (eigenvalues
    +-1/sqrt(k_common + 1), §3.4 Fig. 3).  Group g's nodes get ids
    n + 4g .. n + 4g + 3 (a, b, a', b').  Returns the extended edge list and
    n + 4 n_groups."""
    rng = _rng(seed)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    live = np.zeros(n, bool)
    nl = src != dst
    live[src[nl]] = True
    live[dst[nl]] = True
    cand = np.nonzero(live)[0]
    s_new, d_new = [src], [dst]
    for gi in range(int(n_groups)):
        a, b, la, lb = n + 4 * gi, n + 4 * gi + 1, n + 4 * gi + 2, n + 4 * gi + 3
        common = rng.choice(cand, size=int(k_common), replace=False).astype(np.int64)
        s_new += [np.full(k_common, a), np.full(k_common, b), np.array([a, b], np.int64)]
        d_new += [common, common, np.array([la, lb], np.int64)]
    return np.concatenate(s_new), np.concatenate(d_new), n + 4 * int(n_groups)


def add_parallel_paths(src, dst, n: int, n_groups: int, paths: int, seed: int):
    """Join ``n_groups`` host pairs by ``paths`` new paths of two degree-2
    nodes each (the parallel-path +-1/2 motif of §3.4, Fig. 3).  The 2 n_groups
    hosts are drawn without replacement among the nodes with a non-loop edge
    (pair g = hosts 2g, 2g + 1); path j of pair g uses the new nodes
    n + 2 (g paths + j) and the next one.  Returns the extended edge list and
    the new node count."""
    rng = _rng(seed)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    live = np.zeros(n, bool)
    nl = src != dst
    live[src[nl]] = True
    live[dst[nl]] = True
    hosts = rng.choice(np.nonzero(live)[0], size=2 * int(n_groups), replace=False).astype(np.int64)
    e = np.repeat(hosts[0::2], paths)
    f = np.repeat(hosts[1::2], paths)
    a = n + 2 * np.arange(int(n_groups) * int(paths), dtype=np.int64)
    b = a + 1
    new_src = np.concatenate([src, e, a, b])
    new_dst = np.concatenate([dst, a, b, f])
    return new_src, new_dst, n + 2 * int(n_groups) * int(paths)


def grid2d(nx: int, ny: int):
    """nx x ny grid graph (4-neighbour lattice), node id = y * nx + x: a graph
    with small vertex separators (O(sqrt N)), the case nested dissection (§3.3)
    is made for."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    src = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    dst = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return src, dst, nx * ny


def random_geometric(n: int, radius: float, seed: int):
    """Random geometric graph: n points uniform in the unit square (PCG64
    seed), joined when closer than ``radius`` (found with a cell grid of side
    radius).  Small separators, like road and mesh networks."""
    rng = _rng(seed)
    pts = rng.random((n, 2))
    cells = max(1, int(1.0 / radius))
    cx = np.minimum((pts[:, 0] * cells).astype(np.int64), cells - 1)
    cy = np.minimum((pts[:, 1] * cells).astype(np.int64), cells - 1)
    cell = cy * cells + cx
    order = np.argsort(cell, kind="stable")
    start = np.searchsorted(cell[order], np.arange(cells * cells + 1))
    srcs, dsts = [], []
    r2 = radius * radius
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ny_, nx_ = cy + dy, cx + dx
            ok = (nx_ >= 0) & (nx_ < cells) & (ny_ >= 0) & (ny_ < cells)
            for i in np.nonzero(ok)[0]:
                c = ny_[i] * cells + nx_[i]
                js = order[start[c]:start[c + 1]]
                js = js[js > i]
                if js.size == 0:
                    continue
                d2 = ((pts[js] - pts[i]) ** 2).sum(axis=1)
                js = js[d2 < r2]
                srcs.append(np.full(js.size, i, np.int64))
                dsts.append(js.astype(np.int64))
    if not srcs:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), n
    return np.concatenate(srcs), np.concatenate(dsts), n


def windmill(k: int):
    """Windmill (friendship) graph: k triangles sharing the centre 0; outer
    pair (2t+1, 2t+2) of each triangle are closed twins of degree 2."""
    t = np.arange(k, dtype=np.int64)
    a, b = 2 * t + 1, 2 * t + 2
    return np.concatenate([np.zeros(k, np.int64), np.zeros(k, np.int64), a]), np.concatenate([a, b, b]), 2 * k + 1


# ---------------------------------------------------------------------------
# small deterministic graphs with closed-form spectra (for pins)
# ---------------------------------------------------------------------------

def cycle(n: int):
    """Cycle C_n (n >= 3)."""
    u = np.arange(n, dtype=np.int64)
    return u, (u + 1) % n, n


def path(n: int):
    """Path P_n."""
    u = np.arange(n - 1, dtype=np.int64)
    return u, u + 1, n


def complete(n: int):
    """Complete graph K_n."""
    u, v = np.triu_indices(n, 1)
    return u.astype(np.int64), v.astype(np.int64), n


def star(n_leaves: int):
    """Star K_{1,n}: hub 0, leaves 1..n."""
    v = np.arange(1, n_leaves + 1, dtype=np.int64)
    return np.zeros(n_leaves, np.int64), v, n_leaves + 1


def complete_bipartite(a: int, b: int):
    """K_{a,b}: parts {0..a-1} and {a..a+b-1}."""
    u, v = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return u.ravel().astype(np.int64), v.ravel().astype(np.int64), a + b


def union(graphs):
    """Concatenate graphs [(src, dst, n), ...] into one edge list with global ids.

    Returns (src, dst, node_offset) where graph g owns ids
    [node_offset[g], node_offset[g+1]).
    """
    offs = [0]
    srcs, dsts = [], []
    for s, d, n in graphs:
        srcs.append(np.asarray(s, np.int64) + offs[-1])
        dsts.append(np.asarray(d, np.int64) + offs[-1])
        offs.append(offs[-1] + int(n))
    return (np.concatenate(srcs) if srcs else np.zeros(0, np.int64),
            np.concatenate(dsts) if dsts else np.zeros(0, np.int64), np.asarray(offs, np.int64))


def batch_graphs(count: int, seed: int, n_min: int = 200, n_max: int = 20000):
    """A batch of uneven graphs for the many-small-graphs workload.

    Graph g draws N uniform in [n_min, n_max] and a model uniformly from
    {Erdos-Renyi, Barabasi-Albert with m in [2, 15], Chung-Lu with exponent in
    [2.1, 3.0]}; Erdos-Renyi and Chung-Lu draw a mean degree uniform in [4, 30].
    Yields (src, dst, n, description) per graph.
    """
    rng = _rng(seed)
    for g in range(count):
        n = int(rng.integers(n_min, n_max + 1))
        kind = int(rng.integers(0, 3))
        gseed = int(rng.integers(0, 2**62))
        if kind == 0:
            md = float(rng.uniform(4.0, 30.0))
            s, d, nn = erdos_renyi(n, md / max(n - 1, 1), gseed)
            desc = f"er(n={n},mean_deg={md:.2f})"
        elif kind == 1:
            m = int(rng.integers(2, 16))
            s, d, nn = barabasi_albert(n, m, gseed)
            desc = f"ba(n={n},m={m})"
        else:
            gam = float(rng.uniform(2.1, 3.0))
            md = float(rng.uniform(4.0, 30.0))
            s, d, nn = chung_lu(n, gam, md, gseed)
            desc = f"cl(n={n},gamma={gam:.2f},mean_deg={md:.2f})"
        yield s, d, nn, desc


def _chung_lu_sorted(n: int, gamma: float, mean_degree: float, rng, i0: float = 10.0):
    """Chung-Lu endpoint sampling as in chung_lu, drawn faster: each endpoint
    list is found from sorted uniforms (a sequential search), then the second
    list is randomly permuted.  Given the two endpoint multisets the pairing
    is then uniformly random, as it is for independent pairs, so the edge
    multiset has the same distribution (not the same draws) as chung_lu's.
    Returns int32 endpoints."""
    i = np.arange(n, dtype=np.float64)
    w = (i + i0) ** (-1.0 / (gamma - 1.0))
    w *= mean_degree * n / w.sum()
    m = int(round(n * mean_degree / 2.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(m)
    u.sort()
    src = np.minimum(np.searchsorted(cdf, u, side="right"), n - 1).astype(np.int32)
    u = rng.random(m)
    u.sort()
    dst = rng.permutation(np.minimum(np.searchsorted(cdf, u, side="right"), n - 1).astype(np.int32))
    return src, dst


def chung_lu_twins_member(seed: int, n_min: int, n_max: int):
    """One graph of the Chung-Lu-with-twins family (see chung_lu_twins_family),
    as int32 edge lists (src, dst, n)."""
    rng = _rng(seed)
    n = int(rng.integers(n_min, n_max + 1))
    gam = float(rng.uniform(2.1, 3.0))
    md = float(rng.uniform(5.0, 30.0))
    frac = float(rng.uniform(0.0, 0.1))
    s, d = _chung_lu_sorted(n, gam, md, rng)
    hosts = int(frac * n)
    if hosts > 0:
        live = np.zeros(n, bool)
        nl = s != d
        live[s[nl]] = True
        live[d[nl]] = True
        cand = np.nonzero(live)[0]
        hosts = min(hosts, cand.size)
        h = rng.choice(cand, size=hosts, replace=False).astype(np.int32)
        leaves = n + np.arange(2 * hosts, dtype=np.int32)
        s = np.concatenate([s, np.repeat(h, 2)])
        d = np.concatenate([d, leaves])
        n += 2 * hosts
    return s, d, n


def chung_lu_twins_family(count: int, seed: int, n_min: int = 10_000, n_max: int = 80_000):
    """Training family for the learned reconstruction: Chung-Lu graphs with N
    uniform in [n_min, n_max], exponent uniform in [2.1, 3.0], mean degree
    uniform in [5, 30] (endpoints drawn as in _chung_lu_sorted), plus two
    twin leaves on each of a fraction uniform in [0, 0.1] of N hosts drawn
    among the non-isolated nodes.  Graph k is
    chung_lu_twins_member(seed * 1_000_003 + k, ...), so members can be
    generated independently (in parallel)."""
    for k in range(count):
        yield chung_lu_twins_member(seed * 1_000_003 + k, n_min, n_max)
