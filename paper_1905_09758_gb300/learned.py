"""Learned reconstruction of a graph's spectral density from few noisy moments.

Not part of the paper's method: a small network (``dos_mlp_*``) maps the
Jackson histogram and the first ``m_in`` moments of a cheap KPM run on the
twin-filtered operator P^T H P (§3.4), with the graph's degree statistics
(mean, spread, largest degree) and noise level (N * Nz), to that operator's
density over ``bins`` equal bins of [-1, 1]; the filtered spike at 0 and the r/N scale are
added afterwards exactly as for the plain filtered series.  It is trained on
pairs (cheap run, accurate run: ``m_ref`` moments, ``nz_ref`` probes,
independent seed) computed by the library on graphs of the family it will be
used on.  Plain Jackson-damped KPM (``density_with_spikes``) is its fallback.

This module only sequences calls of the C ABI (argument marshalling and the
training loop's schedule); every computation runs in the library's kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as nd


@dataclass
class Reconstructor:
    """A trained network and the settings its features were made with."""

    net: nd.Mlp
    m_in: int
    nz_in: int
    bins: int
    stats: bool = True  # degree statistics and noise level among the inputs

    @property
    def sizes(self):
        return self.net.sizes


def filtered_operator(src, dst, n_nodes: int, stream=None):
    """CSR handle and twin filter of an edge list (int64 tensors, CUDA or host)."""
    src = torch.as_tensor(src, dtype=torch.int64)
    dst = torch.as_tensor(dst, dtype=torch.int64)
    g = nd.dos_build_csr(src, dst, n_nodes, stream=stream)
    return g, nd.dos_motif_filter(g, stream=stream)


def features(g: nd.Graph, f: nd.Filter | None, m_in: int, nz_in: int, seed: int, bins: int, stats: bool = True,
             stream=None) -> torch.Tensor:
    """Feature row (1, bins + m_in - 1 [+ 4]) of a graph from a cheap filtered
    run (and its degree statistics when ``stats``)."""
    d = nd.dos_moments(g, m_in, nz_in, seed, filter=f, stream=stream)
    h = nd.dos_density(d, bins, stream=stream)
    st = nd.dos_graph_stats(g, nz_in, stream=stream).view(1, 4) if stats else None
    return nd.dos_mlp_features(h.view(1, bins), d.view(1, m_in), m_in, stats=st, stream=stream)


def target(g: nd.Graph, f: nd.Filter | None, m_ref: int, nz_ref: int, seed: int, bins: int,
           stream=None) -> torch.Tensor:
    """Target row (1, bins): the accurate run's filtered density, clipped at 0
    and normalised to unit mass."""
    d = nd.dos_moments(g, m_ref, nz_ref, seed, filter=f, stream=stream)
    h = nd.dos_density(d, bins, stream=stream)
    return nd.dos_hist_normalize(h.view(1, bins), stream=stream)


def training_set(graphs, m_in: int = 50, nz_in: int = 8, m_ref: int = 500, nz_ref: int = 256, bins: int = 200,
                 seed: int = 0, stats: bool = True, stream=None):
    """(X, T) for an iterable of edge lists (src, dst, n_nodes): one row per graph.
    Graph k uses input seed seed + 2k and reference seed seed + 2k + 1."""
    xs, ts = [], []
    for k, (src, dst, n) in enumerate(graphs):
        g, f = filtered_operator(src, dst, n, stream=stream)
        xs.append(features(g, f, m_in, nz_in, seed + 2 * k, bins, stats=stats, stream=stream))
        ts.append(target(g, f, m_ref, nz_ref, seed + 2 * k + 1, bins, stream=stream))
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def training_sets(graphs, m_ins, nz_in: int = 8, m_ref: int = 500, nz_ref: int = 256, bins: int = 200, seed: int = 0,
                  stats: bool = True, stream=None):
    """({m_in: X}, T) for several input sizes at once: one cheap run of
    max(m_ins) moments per graph gives the first m_in moments of each (the
    doubled recurrence's first moments do not depend on how many follow), and
    each X gets the Jackson histogram of its own first m_in moments.  Graph k
    uses input seed seed + 2k and reference seed seed + 2k + 1, as
    training_set."""
    m_ins = sorted(set(int(m) for m in m_ins))
    xs = {m: [] for m in m_ins}
    ts = []
    m_max = m_ins[-1]
    for k, (src, dst, n) in enumerate(graphs):
        g, f = filtered_operator(src, dst, n, stream=stream)
        d = nd.dos_moments(g, m_max, nz_in, seed + 2 * k, filter=f, stream=stream)
        st = nd.dos_graph_stats(g, nz_in, stream=stream).view(1, 4) if stats else None
        for m in m_ins:
            dm = d[:m].contiguous()
            h = nd.dos_density(dm, bins, stream=stream)
            xs[m].append(nd.dos_mlp_features(h.view(1, bins), dm.view(1, m), m, stats=st, stream=stream))
        ts.append(target(g, f, m_ref, nz_ref, seed + 2 * k + 1, bins, stream=stream))
    return {m: torch.cat(v).contiguous() for m, v in xs.items()}, torch.cat(ts).contiguous()


def train(x: torch.Tensor, t: torch.Tensor, m_in: int, nz_in: int, hidden=(512, 512), steps: int = 8000,
          batch: int = 256, lr: float = 1e-3, lr_min: float = 1e-5, seed: int = 0, stream=None,
          resume: Reconstructor | None = None, stop: int | None = None) -> Reconstructor:
    """Adam on minibatches drawn uniformly with replacement, learning rate on a
    cosine schedule from lr to lr_min over `steps` steps.  Whether the rows
    carry the degree statistics is read from their width.  `stop` ends the run
    after that many schedule steps; `resume` (a network saved part-way through
    the same schedule, see save / load) continues it from the Adam step it
    had reached, so an interrupted run ends where an uninterrupted one would."""
    bins = t.shape[1]
    gen = torch.Generator().manual_seed(seed)
    idx = torch.randint(0, x.shape[0], (steps, batch), generator=gen, dtype=torch.int32).to(x.device)
    if resume is not None:
        net = resume.net
        start = nd.dos_mlp_get_state(net)["step"]
    else:
        net = nd.dos_mlp_create([x.shape[1], *hidden, bins], seed=seed)
        start = 0
    for s in range(start, steps if stop is None else min(stop, steps)):
        rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * s / steps))
        nd.dos_mlp_train_step(net, x, t, rate, idx=idx[s], stream=stream)
    return Reconstructor(net, m_in, nz_in, bins, stats=x.shape[1] == bins + m_in - 1 + 4)


def save(rec: Reconstructor, path, with_optimizer: bool = True) -> None:
    """Write a network and the settings of its features to `path` (numpy
    .npz): layer sizes, m_in, nz_in, bins, whether the degree statistics are
    inputs, the parameters and, with_optimizer, Adam's moments and step count
    (what train(resume=...) needs to continue)."""
    st = nd.dos_mlp_get_state(rec.net)
    arrays = {"sizes": np.asarray(rec.sizes, np.int64),
              "meta": np.asarray([rec.m_in, rec.nz_in, rec.bins, int(rec.stats)], np.int64),
              "params": st["params"].cpu().numpy()}
    if with_optimizer:
        arrays.update(m=st["m"].cpu().numpy(), v=st["v"].cpu().numpy(), step=np.asarray(st["step"], np.int64))
    np.savez(path, **arrays)


def load(path) -> Reconstructor:
    """A network written by save, on the current CUDA device."""
    with np.load(path) as z:
        net = nd.dos_mlp_create([int(v) for v in z["sizes"]])
        params = torch.from_numpy(z["params"])
        if "m" in z:
            nd.dos_mlp_set_state(net, {"params": params, "m": torch.from_numpy(z["m"]), "v": torch.from_numpy(z["v"]),
                                       "step": int(z["step"])})
        else:
            nd.dos_mlp_set_params(net, params.to(torch.device("cuda", torch.cuda.current_device())))
            torch.cuda.synchronize()
        m_in, nz_in, bins, stats = (int(v) for v in z["meta"])
    return Reconstructor(net, m_in, nz_in, bins, stats=bool(stats))


def reconstruct(rec: Reconstructor, g: nd.Graph, f: nd.Filter | None, seed: int, count_isolated: bool = True,
                stream=None) -> torch.Tensor:
    """Spectral histogram (float64 CUDA, rec.bins) of the whole graph: the
    network's density of the filtered operator scaled by r / N_total, plus the
    eigenvalues the filter removed (and isolated nodes at 0) as point masses."""
    x = features(g, f, rec.m_in, rec.nz_in, seed, rec.bins, stats=rec.stats, stream=stream)
    p = nd.dos_mlp_forward(rec.net, x, stream=stream)
    scale, spikes = nd.filtered_scale_and_spikes(g, f, count_isolated)
    return nd.dos_hist_assemble(p, scale=scale, spikes=spikes, stream=stream)[0]
