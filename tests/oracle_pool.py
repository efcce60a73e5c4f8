"""Oracle runs split over probe columns in worker processes (test
infrastructure).

The trace estimator of Eq. (11) is a sum over probes, mu_m = sum_j z_j^T
T_m(H) z_j, and the twin projection Z_r = P P^T Z of §3.4 acts column by
column, so the oracle's moments of a probe block are the sum of its moments
of column subsets.  Each worker rebuilds the seeded graph and the oracle CSR
itself (nothing crosses from the library) and returns the oracle's moments of
its columns.  The pool uses the spawn start method, so it is safe after CUDA
has been initialised in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _graph(spec):
    import synthgraphs as sg

    kind = spec[0]
    if kind == "chung_lu_twins":
        _, n_base, gamma, mean_deg, n_hosts, seed = spec
        s, d, n = sg.chung_lu(n_base, gamma, mean_deg, seed)
        return sg.add_twin_leaves(s, d, n, n_hosts, seed + 1)
    raise ValueError(kind)


def _doubled_chunk(args):
    spec, seed, nz, cols, m, filtered = args
    import oracle

    s, d, n = _graph(spec)
    ref = oracle.build_csr(s, d, n)
    z = oracle.probes(seed, ref.old_id, nz)
    r = ref.n
    if filtered:
        cid, removed = oracle.twin_classes(ref)
        z = oracle.project_probes(z, cid)
        r = ref.n - removed
    return oracle.kpm_doubled(ref, z[:, cols], m), r


def workers() -> int:
    return max(1, min(16, len(os.sched_getaffinity(0))))


def doubled_moments(spec, seed: int, nz: int, m: int, filtered: bool) -> np.ndarray:
    """Normalised doubled-KPM moments d_m = mu_m / (r Nz) of the graph `spec`
    with the first nz probes of `seed`, the probe columns split over worker
    processes (oracle.kpm_doubled on each subset, summed)."""
    w = min(workers(), nz)
    chunks = [list(c) for c in np.array_split(np.arange(nz), w)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(w) as pool:
        parts = pool.map(_doubled_chunk, [(spec, seed, nz, c, m, filtered) for c in chunks])
    mu = np.sum([p[0] for p in parts], axis=0)
    r = parts[0][1]
    return mu / (r * nz)
