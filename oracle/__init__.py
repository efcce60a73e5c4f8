"""Plain FP64 CPU oracle for the network density-of-states method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library
(``paper_1905_09758_gb300``): it re-derives every quantity from the paper's
definitions, in float64, with numpy/scipy primitives (a sort, a sparse
matrix-vector product, a dense symmetric eigensolver) as its only building
blocks.

Every function cites the passage it follows (Dong, Benson, Bindel, "Network
Density of States", KDD 2019).  Readings of passages that are silent or
garbled are stated where they are used.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):

* ``splitmix64`` / ``probes``      -- pinned to the generator's published outputs.
* ``build_csr``                    -- pinned to brute-force adjacency sets.
* ``dense_h``, ``exact_moments``,
  ``exact_ldos``                   -- pinned to closed-form spectra (K_n, C_n,
                                      K_{1,n}, K_{a,b}, bipartite symmetry,
                                      tr T_1 and tr T_2 identities).
* ``kpm_direct``, ``kpm_doubled``  -- pinned to the exact moments (identity
                                      probes give tr T_m(H) exactly) and to each
                                      other.
* ``twin_classes``, ``project_probes``
                                   -- pinned by stars, K_{a,b}, eigenvalue counts
                                      at 0 and the spectrum of P^T H P.
* ``closed_twin_classes``, ``pendant_twin_classes``, ``parallel_path_classes``,
  ``motif_classes``
                                   -- pinned by K_n (one class, -1/(n-1)), windmill
                                      graphs (-1/2), disjointness of the open and
                                      closed relations, P5's closed-form spectrum,
                                      spiders (+-1/sqrt 2), Fig. 3's degree-4 pendant
                                      twins (+-1/2), theta graphs (+-1/2), all motifs
                                      together, invariance of the class-
                                      constant subspace and the spectrum of P^T H P.
* ``jackson``, ``bin_integrals``,
  ``histogram``                    -- pinned by g_0 = 1, kernel positivity,
                                      unit mass, and independent quadrature.
* ``lanczos``, ``gauss_rules``, ``gql_moments``, ``gql_histogram``
                                   -- pinned by Gauss exactness (the rule's Chebyshev
                                      moments equal the KPM moments of the same probes
                                      up to degree 2M - 1), K_n and C_n closed forms,
                                      unit weights and the PDOS of e_k probes.
* ``operator_matrix``, ``gershgorin_interval``, ``exact_operator_moments``,
  ``kpm_operator``                 -- pinned by closed-form spectra of A and L (K_n,
                                      C_n, stars), Gershgorin containment, and identity
                                      probes giving the exact traces.
* ``motif_spikes``                 -- pinned by K_n, star and P5 closed forms for A and L, and by
                                      spec(X) = spec(P^T X P) plus the spikes for all four
                                      operators on a graph with every motif.
* ``ritz_bounds``, ``spectral_interval``, ``lanczos`` on A and L
                                   -- pinned by K_n and star closed forms (the Krylov
                                      space is exhausted: the interval is the exact
                                      spectrum), containment of the dense spectrum,
                                      the Ritz bound's failure before convergence,
                                      and tightness against Gershgorin on hub graphs.
* ``cheb_coeffs``, ``trace_fn``, ``diag_fn``, ``ldos_operator``, ``exact_fn_trace``,
  ``exact_fn_diag``, ``fn_values``
                                   -- pinned by the Bessel (exp) and geometric
                                      (resolvent) closed forms of the coefficients, the
                                      Estrada index of K_n and stars, subgraph and
                                      resolvent centralities of stars, the heat kernel
                                      trace of a star's Laplacian, scipy's expm, and
                                      identity probes giving the exact diagonal.
* ``mlp_*``                        -- pinned by central finite differences.
"""
from .kpm import *  # noqa: F401,F403
from .kpm import __all__ as _kpm_all
from .gql import *  # noqa: F401,F403
from .gql import __all__ as _gql_all
from .mlp import *  # noqa: F401,F403
from .mlp import __all__ as _mlp_all
from .operators import *  # noqa: F401,F403
from .operators import __all__ as _op_all
from .functions import *  # noqa: F401,F403
from .functions import __all__ as _fn_all

__all__ = list(_kpm_all) + list(_gql_all) + list(_op_all) + list(_fn_all) + list(_mlp_all)
