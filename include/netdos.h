/*
 * netdos.h -- C ABI of the GB300 network density-of-states library.
 *
 * The library computes the stochastic Chebyshev (kernel polynomial method,
 * KPM) moments of the normalized adjacency H = D^{-1/2} A D^{-1/2} of an
 * undirected graph, the per-node (local / pointwise) moments, the twin-motif
 * filter and the damped spectral histogram, following Dong, Benson, Bindel,
 * "Network Density of States", KDD 2019 (§2.1 graph operators, §2.2 DOS and
 * LDOS, §3.1 KPM, §3.4 motif filtering, §4.1 Jackson damping).
 *
 * Conventions for every entry point:
 *  - Return value: DOS_OK (0) or a dos_status code; nothing aborts and no C++
 *    exception crosses the ABI.  dos_last_error() returns a thread-local text
 *    for the last failure on the calling thread.
 *  - Pointers marked [device] are CUDA device pointers owned by the caller;
 *    [host] are host pointers owned by the caller.  Handles (dos_graph_t,
 *    dos_filter_t) are owned by the library and released by *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on that stream; calls that return scalars to
 *    the host synchronise it.  A handle must not be used from two streams
 *    concurrently.
 *  - Node numbering: the library compacts away nodes without edges (their
 *    eigenvalue is 0, see dos_density's spikes).  "Compact id" i in [0, N)
 *    is the i-th non-isolated node in increasing original id; old_id[i] is
 *    its original id.  All per-node outputs use compact ids.
 *  - Probes are Rademacher: entry (i, j) for the node with original id o is
 *    +1 if bit (j & 63) of SplitMix64(seed)[((j >> 6) << 32) | o] is 0, else
 *    -1, where SplitMix64(seed)[n] = mix(seed + (n + 1) * 0x9E3779B97F4A7C15)
 *    (Steele, Lea, Flood, OOPSLA 2014).  The paper's probes are i.i.d. with
 *    mean 0 and variance 1 (§3.1); these are such probes.
 */
#ifndef NETDOS_H
#define NETDOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dos_graph_s* dos_graph_t;
typedef struct dos_filter_s* dos_filter_t;
typedef struct dos_mlp_s* dos_mlp_t;

enum dos_status {
  DOS_OK = 0,
  DOS_EINVAL = 1,    /* invalid argument (ids out of range, M < 1, Nz < 1, ...) */
  DOS_ENOMEM = 2,    /* device allocation failed */
  DOS_ECUDA = 3,     /* a CUDA runtime call failed; see dos_last_error() */
  DOS_ETIMEOUT = 4,  /* a bounded device wait gave up */
  DOS_EOVERFLOW = 5  /* size beyond the int32 / int64 index range of a path */
};

/* Storage precision of the probe blocks T_m(H) Z.  Arithmetic is FP32 and
 * the moment reductions are FP64 in every mode. */
enum dos_prec { DOS_FP32 = 0, DOS_BF16 = 1, DOS_FP16 = 2 };

/* Damping of the Chebyshev series in dos_density. */
enum dos_kernel { DOS_KERNEL_NONE = 0, DOS_KERNEL_JACKSON = 1 };

/* Flags of dos_build_csr. */
enum dos_build_flags {
  DOS_INPUT_HOST = 1,    /* src/dst are host pointers: page-locked ones are read
                            in place through their device mapping, others are
                            copied to device temporaries */
  DOS_ORDER_BY_CLASS = 2 /* the kernels' row order keeps the node numbering
                            inside each degree class (see dos_build_csr) */
};

/* Instrumentation, not in the paper. Library version as MAJOR*10000 +
 * MINOR*100 + PATCH. */
int dos_version(void);

/* Error reporting, not in the paper. Thread-local text describing the last
 * failed call on this thread ("" if none). */
const char* dos_last_error(void);

/*
 * dos_build_csr -- undirected edge list -> CSR of A, degrees, D^{-1/2}.
 * Paper: §2.1 (A, D and the normalized adjacency D^{-1/2} A D^{-1/2}).
 *   src, dst   [device, or host with DOS_INPUT_HOST] int64[n_edges]: edge
 *              endpoints, original ids in [0, n_nodes).  Each entry is one
 *              undirected edge; repeated pairs collapse to one edge of
 *              weight 1 and self-loops (u == v) are dropped.
 *   n_edges    >= 0.   n_nodes in [0, 2^31 - 1].
 *   out        receives the graph handle (device memory owned by the library).
 * Column indices are int32 and row offsets int64, so nnz (2 x undirected
 * edges) may exceed 2^31; n_edges <= 2^40.
 * Row order of the step kernels (a project addition, not in the paper; a
 * relabelling, so moments and densities do not depend on it beyond FP
 * rounding, and LDOS rows are returned by compact id):
 * by default degree-descending, so rows processed together have similar
 * degrees.  With DOS_ORDER_BY_CLASS only the three degree classes (>= 2048,
 * >= 64, the rest) are separated and each keeps the node numbering: for
 * graphs numbered so that neighbours have nearby ids (meshes, road networks,
 * a bandwidth-reducing order), whose gathers then stay in L2.
 * Errors: DOS_EINVAL (negative sizes, endpoint out of range -- detected on
 * the device and reported after a stream sync, unknown flags), DOS_ENOMEM,
 * DOS_ECUDA.
 * Synchronises `stream` (the node count is needed on the host).
 */
int dos_build_csr(const int64_t* src, const int64_t* dst, int64_t n_edges,
                  int64_t n_nodes, uint32_t flags, void* stream,
                  dos_graph_t* out);

/* §2.1 (the graph and its compacted node set). Sizes of a built graph [host
 * outputs; any may be NULL]: N = non-isolated nodes, nnz = stored nonzeros (2
 * x undirected edges), n_isolated = nodes dropped for having no edge,
 * n_original = n_nodes given to dos_build_csr. */
int dos_graph_info(dos_graph_t g, int64_t* n, int64_t* nnz,
                   int64_t* n_isolated, int64_t* n_original);

/*
 * §2.1 (A in CSR, degrees, D^{-1/2}).
 * dos_graph_export -- copy the CSR (compact ids) to caller buffers [device].
 *   row_ptr int64[N+1], col int32[nnz] (ascending within each row),
 *   deg int32[N], inv_sqrt_deg double[N] = 1/sqrt(deg) (IEEE, correctly
 *   rounded), inv_sqrt_deg32 float[N] = (float) of that, old_id int32[N].
 *   Any pointer may be NULL to skip that array.  Stream-ordered.
 */
int dos_graph_export(dos_graph_t g, int64_t* row_ptr, int32_t* col,
                     int32_t* deg, double* inv_sqrt_deg,
                     float* inv_sqrt_deg32, int32_t* old_id, void* stream);

void dos_graph_destroy(dos_graph_t g);

/*
 * dos_motif_filter -- find the lambda = 0 twin motif classes.
 * Paper: §3.4 (Fig. 3a: nodes with identical neighbourhoods give localized
 * eigenvectors with eigenvalue 0; detection by hashing; filtering by the
 * projected probes Z_r = P P^T Z).  Classes are the exact relation the hash
 * detects: nodes i != j of degree >= 1 with N(i) = N(j) as sets; hash
 * collisions are resolved by comparing neighbour lists, so the result is
 * deterministic and exact.
 *   out  receives the filter handle.  Synchronises `stream`.
 * Errors: DOS_EINVAL (g NULL), DOS_ENOMEM, DOS_ECUDA.
 */
int dos_motif_filter(dos_graph_t g, void* stream, dos_filter_t* out);

/* Motif sets of dos_motif_filter_ex (bit mask). */
enum {
  DOS_MOTIF_OPEN_TWINS = 1,   /* N(i) = N(j): eigenvalue 0 (Fig. 3a) */
  DOS_MOTIF_CLOSED_TWINS = 2, /* N[i] = N[j] (adjacent, degree d): eigenvalue -1/d */
  DOS_MOTIF_PENDANT_TWINS = 4, /* degree-d nodes equal but for one leaf each: +-1/sqrt(d) */
  DOS_MOTIF_PARALLEL_PATHS = 8 /* >= 2 paths E - a - b - F of degree-2 nodes: +-1/2 */
};

/*
 * dos_motif_filter_ex -- twin-motif classes for a set of motifs.
 * Paper: §3.4 (Fig. 3: motifs with localized eigenvectors; detection by
 * hashing; filtering by Z_r = P P^T Z).  Closed twins are nodes with equal
 * closed neighbourhoods N[i] = N(i) + {i}; they are adjacent, share the degree
 * d, and each class of size c carries c - 1 eigenvalues -1/d on the vectors
 * e_i - e_j (d = 2: the triangle with two degree-2 nodes, -1/2; degree m:
 * the -1/m motif).  Pendant twins are nodes of degree d >= 2 with exactly one
 * leaf neighbour each and equal neighbourhoods apart from it (d = 2: pendant
 * 2-paths u - a - a'; d = 4: the +-1/2 motif); a class of c carries c - 1
 * eigenvalues at each of +-1/sqrt(d) on vectors summing to zero over the
 * nodes and over their leaves, which become two classes.  Parallel paths
 * are c >= 2 paths E - a - b - F through degree-2 nodes between the same
 * hosts E != F of degree >= 3 (Fig. 3's first +-1/2 drawing): the nodes next
 * to each host form a class, c - 1 eigenvalues at each of +-1/2.
 * The relations are disjoint, so all classes are filtered by one class-mean
 * projection; dos_filter_info's removed counts all of them, and
 * dos_filter_spikes lists the removed eigenvalues.  Hash collisions are
 * resolved by exact comparison.
 *   motifs  any nonzero OR of the DOS_MOTIF_* values.
 *   out     receives the filter handle.  Synchronises `stream`.
 * Errors: DOS_EINVAL (g NULL, empty or unknown motif set), DOS_ENOMEM,
 * DOS_ECUDA.  dos_motif_filter(g, ...) = dos_motif_filter_ex(g,
 * DOS_MOTIF_OPEN_TWINS, ...).
 */
int dos_motif_filter_ex(dos_graph_t g, uint32_t motifs, void* stream,
                        dos_filter_t* out);

/* §3.4, Fig. 3 (motif eigenvalues). Removed eigenvalues [host]: up to
 * `capacity` pairs (lambda, count) in ascending lambda (0 for open twins, -1/d
 * per degree d with closed twins, +-1/sqrt(d) per degree d with pendant twins,
 * +-1/2 for parallel paths; equal values of different motifs are one entry);
 * *n_spikes (may be NULL) receives the total number of pairs. Errors:
 * DOS_EINVAL. */
int dos_filter_spikes(dos_filter_t f, double* spikes, int capacity,
                      int* n_spikes);

/* §3.4 (filtered eigenvalue counts). Filter summary [host outputs; any may be
 * NULL]: removed = sum over classes of (size - 1) = number of eigenvalues at 0
 * the filter takes out, n_classes = classes of size >= 2, r = N - removed. */
int dos_filter_info(dos_filter_t f, int64_t* removed, int64_t* n_classes,
                    int64_t* r);

/* §3.4 (motif classes). class_id [device] int32[N]: the smallest compact id in
 * each node's class (a node's own id if it has no twin).  Stream-ordered. */
int dos_filter_export(dos_filter_t f, int32_t* class_id, void* stream);

void dos_filter_destroy(dos_filter_t f);

/*
 * dos_moments -- stochastic DOS moments d_0 .. d_{M-1}.
 * Paper: §3.1, Eq. (6) (Chebyshev recurrence on H), Eq. (9) (d_m = tr T_m(H)
 * / N) and Eq. (11) (trace estimator with Nz probes).  The recurrence runs
 * floor(M/2) sparse products: with V_k = T_k(H) Z, per probe
 *   mu_{2k}   = 2 <V_k, V_k>     - <V_0, V_0>
 *   mu_{2k+1} = 2 <V_{k+1}, V_k> - <V_1, V_0>.
 *   f       NULL for plain probes, or a filter from dos_motif_filter on the
 *           same graph: then Z is replaced by Z_r = P P^T Z (class means,
 *           §3.4) and the moments are those of the reduced operator P^T H P.
 *   M >= 1, Nz >= 1, prec a dos_prec.
 *   d_out   [device] double[M]: d_m = mu_m / (r * Nz), r = N without a
 *           filter, r = N - removed with one.
 * Scratch: two probe blocks of N x Nz elements of the storage precision and a
 * small FP64 partial-sum array, allocated stream-ordered on `stream` and
 * released before return.  Stream-ordered (does not synchronise).
 * Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_moments(dos_graph_t g, dos_filter_t f, int M, int Nz, uint64_t seed,
                int prec, double* d_out, void* stream);

/* Graph operators of dos_moments_op (§2.1). */
enum {
  DOS_OP_NORMALIZED_ADJACENCY = 0, /* H = D^{-1/2} A D^{-1/2}, spectrum in [-1, 1] */
  DOS_OP_ADJACENCY = 1,            /* A */
  DOS_OP_LAPLACIAN = 2,            /* L = D - A */
  DOS_OP_NORMALIZED_LAPLACIAN = 3  /* I - H, spectrum in [0, 2] */
};

/*
 * dos_moments_op -- DOS moments of another graph operator X.
 * Paper: §2.1 (the operators), Eq. (5) (an interval [a, b] holding the
 * spectrum is mapped onto [-1, 1]: X~ = (X - c) / r, c = (a + b) / 2,
 * r = (b - a) / 2), then §3.1 as dos_moments on X~ (doubling, Eq. (6), (9),
 * (11)).  d_m = tr T_m(X~) / N estimated from Nz Rademacher probes (the
 * probes of dos_moments for the same seed).
 *   op   DOS_OP_*.  H: [a, b] = [-1, 1] (= dos_moments without a filter);
 *        I - H: [0, 2], its moments are (-1)^m those of H; the random-walk
 *        matrix D^{-1} A = D^{-1/2} H D^{1/2} has the spectrum of H.
 *        A and D - A: [a, b] = [lo, hi] if lo < hi, else the Gershgorin
 *        interval [-d_max, d_max] (A) or [0, 2 d_max] (D - A).
 *   d_out        [device] double[M]
 *   interval_out [host] double[2] receives [a, b] (may be NULL).
 *   prec as dos_moments.  Stream-ordered.
 * Errors: DOS_EINVAL (unknown operator, ...), as dos_moments otherwise.
 */
int dos_moments_op(dos_graph_t g, int op, double lo, double hi, int M, int Nz,
                   uint64_t seed, int prec, double* d_out,
                   double* interval_out, void* stream);

/*
 * ldos_moments -- per-node (pointwise) moments, and the DOS moments from them.
 * Paper: §2.2 Eq. (2) (LDOS), Eq. (10) (d_mk = T_m(H)_kk), Eq. (12) (diagonal
 * estimator E[z o Hz] = diag H).  Direct recurrence, M - 1 sparse products:
 *   C[m][k] = (1/Nz) sum_j z_kj (T_m(H) z_j)_k.
 *   C_out  [device] float[M * N], MOMENT-MAJOR: C_out[m * N + k] is moment m
 *          of compact node k (i.e. a column-major N x M matrix).
 *   d_out  [device] double[M] or NULL: d_m = (1/(N Nz)) sum_k sum_j
 *          z_kj (T_m(H) z_j)_k, the same estimator as dos_moments without a
 *          filter, from the direct recurrence.
 * Probes are never projected here (a projected probe would estimate the
 * diagonal of P P^T T_m(H) P P^T instead).  Scratch as for dos_moments, plus,
 * when the plan has several probe tiles, a buffer of up to 32 moments x tiles
 * x N floats (at most 256 MB) in which each tile's contribution is stored and
 * then summed in a fixed order, so C_out is bitwise reproducible.
 * Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int ldos_moments(dos_graph_t g, int M, int Nz, uint64_t seed, int prec,
                 float* C_out, double* d_out, void* stream);

/* Layouts of the N x M LDOS matrix (ldos_moments_ex). */
enum dos_layout {
  DOS_MOMENT_MAJOR = 0, /* C_out[m * N + k]: one contiguous row per moment */
  DOS_NODE_MAJOR = 1    /* C_out[k * M + m]: N x M row-major, one row per node */
};

/*
 * ldos_moments_ex -- ldos_moments with a choice of output layout.
 * Paper: §2.2 Eq. (2), Eq. (10), Eq. (12), as ldos_moments; Algorithm 1's
 * output is the N x M matrix of per-node moments, which DOS_NODE_MAJOR gives
 * row-major.  The steps produce one moment for all nodes at a time, so with
 * DOS_NODE_MAJOR (or with several probe tiles) they write a scratch of up to
 * 32 moments and a fold kernel sums the tiles in a fixed order and writes
 * the chunk in the layout (through a shared-memory transpose for
 * DOS_NODE_MAJOR).  Values are identical in both layouts.
 *   layout  DOS_MOMENT_MAJOR or DOS_NODE_MAJOR;  C_out [device] float[M * N].
 *   Other arguments, scratch and errors as ldos_moments (DOS_EINVAL for an
 *   unknown layout).
 */
int ldos_moments_ex(dos_graph_t g, int M, int Nz, uint64_t seed, int prec,
                    int layout, float* C_out, double* d_out, void* stream);

/*
 * ldos_moments_op -- ldos_moments on another operator X (§2.1), mapped by
 * Eq. (5) as in dos_moments_op: C[m][k] = (1/Nz) sum_j z_kj (T_m(X~) z_j)_k,
 * the diagonal estimator of Eq. (12) on X~ (C[m][k] estimates T_m(X~)_kk).
 *   op, lo, hi, interval_out as dos_moments_op (I - H: odd rows negated).
 *   C_out, d_out as ldos_moments.  FP32 storage.  Stream-ordered.
 * Errors: DOS_EINVAL (unknown operator, ...), as ldos_moments otherwise.
 */
int ldos_moments_op(dos_graph_t g, int op, double lo, double hi, int M, int Nz,
                    uint64_t seed, float* C_out, double* d_out,
                    double* interval_out, void* stream);

/* Flags of dos_density / dos_density_weights. */
enum dos_density_flags {
  DOS_DENSITY_COUNT_ISOLATED = 1 /* nodes without edges count as eigenvalue 0 */
};

/*
 * dos_density -- damped spectral histogram of a graph from its moments.
 * Paper: §2.2 (spectral histogram on equal bins), Eq. (7)-(8) (dual Chebyshev
 * basis, expansion of the DOS), §4.1 (Jackson damping; the factors are the
 * Jackson kernel of the KPM literature for M terms:
 * g_m = [(M-m+1) cos(pi m/(M+1)) + sin(pi m/(M+1)) cot(pi/(M+1))]/(M+1)),
 * §3.4 (the filtered density: the reduced operator's series weighted by
 * r / N plus the removed eigenvalues as point masses).
 *   d        [device] double[M] moments d_0 .. d_{M-1} (of P^T H P when f is
 *            given, i.e. dos_moments with that filter).
 *   n_bins   B >= 1 equal bins over [-1, 1].  M <= 2^20.
 *   kernel   DOS_KERNEL_JACKSON or DOS_KERNEL_NONE (g_m = 1).
 *   g, f     NULL, NULL: the plain series (scale 1, no point masses).
 *            Otherwise the whole graph's density: g the graph (may be NULL
 *            when f is given: f's graph), f a filter of g or NULL.  With
 *            N_total = N + n_isolated (flag DOS_DENSITY_COUNT_ISOLATED) or N,
 *            r = N - removed (N without a filter): the series part is scaled
 *            by r / N_total and every eigenvalue the filter removed (and the
 *            isolated nodes, at 0, when counted) is a point mass count /
 *            N_total (dos_density_weights returns these numbers).
 *   flags    0 or DOS_DENSITY_COUNT_ISOLATED.
 *   hist_out [device] double[B]: bin b gets
 *            scale * (g_0 d_0 I_0b + 2 sum_{m>=1} g_m d_m I_mb) + spikes,
 *            I_mb = integral over bin b of T_m(x) / (pi sqrt(1 - x^2)) dx; a
 *            point mass within 1e-9 of an interior bin edge splits evenly
 *            between the two bins, +-1 go to the end bins.
 * Stream-ordered.  Errors: DOS_EINVAL (null pointer, sizes, a filter of
 * another graph, more than 64 distinct point masses).
 */
int dos_density(const double* d, int M, int n_bins, int kernel,
                dos_graph_t g, dos_filter_t f, uint32_t flags,
                double* hist_out, void* stream);

/* §3.4 (filtered density weights), §2.2. The numbers dos_density uses for
 * (g, f, flags) [host outputs, any may be NULL]: scale_out = r / N_total, and
 * up to `capacity` pairs (lambda, mass) in spikes_out[2 * capacity] in
 * ascending lambda, mass = count / N_total; *n_spikes the number of pairs.
 * g may be NULL when f is given.  Errors: DOS_EINVAL. */
int dos_density_weights(dos_graph_t g, dos_filter_t f, uint32_t flags,
                        double* scale_out, double* spikes_out, int capacity,
                        int* n_spikes);

/* §2.2, Eq. (7)-(8), §4.1 with an explicit weight: dos_density's series times
 * `scale` plus the point masses (lambda, mass) of spikes [host double[2 *
 * n_spikes], n_spikes <= 64, NULL if 0], placed as in dos_density.
 * Stream-ordered.  Errors: DOS_EINVAL. */
int dos_density_raw(const double* d, int M, int n_bins, int kernel,
                    double scale, const double* spikes, int n_spikes,
                    double* hist_out, void* stream);

/*
 * A project addition (not in the paper): the paper has no counterpart to this
 * entry point; the computation it runs is dos_moments'.
 * dos_moments_noalloc -- dos_moments (FP32 storage, no filter) for callers
 * that cannot allocate device memory.
 * Who needs it: a caller whose framework allocator already holds nearly all
 * device memory (a fresh cudaMalloc would fail or force the framework to
 * drop its cache), or a latency-bound caller for which cudaMalloc/cudaFree,
 * which may synchronise the device, are not acceptable.  This call allocates
 * nothing: its scratch (two probe blocks of N x Nz_pad floats and the FP64
 * moment partials) lives in one static device array of 16 MiB that every GPU
 * loading the library holds until the process exits.
 *   g, M, Nz, seed, d_out, stream: as for dos_moments (d_out [device]
 *   double[M], caller-allocated).  Results are bitwise equal to dos_moments'
 *   with f = NULL and prec = DOS_FP32: the same kernels, plan and fixed
 *   reduction order on a different scratch address.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array and its contents persist between
 * calls; each call clears what must start at zero.  Calls that overlap on
 * the GPU (other streams or threads) race on the shared array.
 * Errors: DOS_EINVAL when the graph, M and Nz need more than the 16 MiB
 * scratch (the message states both sizes; use dos_moments), or for invalid
 * arguments as in dos_moments; DOS_ECUDA.
 */
int dos_moments_noalloc(dos_graph_t g, int M, int Nz, uint64_t seed,
                        double* d_out, void* stream);

/*
 * dos_pdos_nd -- exact PDOS moments by nested dissection.
 * Paper: §3.3 (block recurrence for T_m(H) on a partition tree, Eq. (13)-(14))
 * and Algorithm 1.  C_out[m * N + k] = T_m(H)_kk (compact ids), m < M,
 * computed exactly up to FP32 rounding, without probes.  The partition tree
 * is built on the host by recursive bisection with BFS level sets as vertex
 * separators (partitions of at most leaf_size nodes are leaves); the cost and
 * memory are the sum over tree nodes of |partition| x |separator| (three
 * FP32 buffers of that many entries), small when the graph has small
 * separators (meshes, road-like and geometric graphs) and prohibitive when it
 * has not (expanders, power-law graphs).
 *   leaf_size    >= 1 (e.g. 64)
 *   max_entries  refuse (DOS_ENOMEM) when the block entries exceed this;
 *                <= 0: no limit
 *   C_out [device] float[M * N]
 *   stats [host] int64[4] or NULL: tree nodes, depth levels, block entries,
 *                largest separator.
 * Stream-ordered after the partitioning (which synchronises `stream`).
 * Errors: DOS_EINVAL, DOS_ENOMEM (too many block entries), DOS_ECUDA.
 */
int dos_pdos_nd(dos_graph_t g, int M, int leaf_size, double max_entries,
                float* C_out, int64_t* stats, void* stream);

/* ---------------------------------------------------------------------
 * Gauss quadrature and Lanczos (GQL), the second estimator of §3.2.
 * --------------------------------------------------------------------- */

/*
 * dos_lanczos -- M Lanczos steps on H from each of Nz Rademacher probes (the
 * probes of dos_moments for the same seed), FP32 vectors, FP64 reductions,
 * no reorthogonalisation.  Paper: §3.2 (H Z_M = Z_M Gamma_M + r_M e_M^T).
 *   alpha_out [device] double[Nz * M]: alpha_out[p * M + k] = alpha_k of probe
 * p
 *   beta_out  [device] double[Nz * M]: beta_out[p * M + k] = ||w_{k+1}||, the
 *             coupling of steps k and k + 1 (the last one is the residual)
 *   steps_out [device] int32[Nz]: steps run; a probe stops early when
 *             beta_k <= 1e-5 (its Krylov space is exhausted; below 1e-5 ||H||
 *             the FP32 residual is rounding noise); entries past its steps
 *             are 0.
 *   M in [1, 4096], Nz in [1, 128].  Stream-ordered.
 * Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_lanczos(dos_graph_t g, int M, int Nz, uint64_t seed, double* alpha_out,
                double* beta_out, int32_t* steps_out, void* stream);

/*
 * dos_lanczos_op -- dos_lanczos on another operator X of §2.1: op =
 * DOS_OP_NORMALIZED_ADJACENCY (H, = dos_lanczos), DOS_OP_ADJACENCY (A) or
 * DOS_OP_LAPLACIAN (D - A), unscaled, on the non-isolated nodes.  Outputs as
 * dos_lanczos, in the units of X; a probe stops when beta_k <= 1e-5 x the
 * Gershgorin bound of ||X|| (1, d_max, 2 d_max).  Stream-ordered.
 * Errors: DOS_EINVAL (op DOS_OP_NORMALIZED_LAPLACIAN or unknown, ...), as
 * dos_lanczos otherwise.
 */
int dos_lanczos_op(dos_graph_t g, int op, int M, int Nz, uint64_t seed,
                   double* alpha_out, double* beta_out, int32_t* steps_out,
                   void* stream);

/* Margins of dos_spectral_interval. */
enum {
  DOS_BOUND_RESIDUAL = 0, /* theta -+ beta_M: safe after a few steps */
  DOS_BOUND_RITZ = 1      /* theta -+ beta_M |s_M|: tight once converged */
};

/* §3.2 (Lanczos on X), Eq. (5). Per-probe bounds of dos_spectral_interval from
 * Lanczos coefficients as produced by dos_lanczos_op [device]: bounds_out[2p]
 * = theta_min - r, bounds_out[2p + 1] = theta_max + r [device double[2 Nz]],
 * theta the extreme eigenvalues of probe p's tridiagonal (bisection), r as
 * chosen by bound (DOS_BOUND_*).  Stream-ordered.  Errors: DOS_EINVAL. */
int dos_ritz_bounds(const double* alpha, const double* beta,
                    const int32_t* steps, int M, int Nz, int bound,
                    double* bounds_out, void* stream);

/*
 * dos_spectral_interval -- an interval [a, b] holding the spectrum of X, for
 * the map onto [-1, 1] of Eq. (5) (dos_moments_op), much tighter than the
 * Gershgorin interval on graphs with hubs.  M Lanczos steps on X (H for
 * I - H) from Nz probes (§3.2's recurrence); each probe gives
 * [theta_min - r, theta_max + r], its extreme Ritz values widened by
 *   DOS_BOUND_RESIDUAL  r = beta_M, the residual norm of the last step (on
 *                       Nz >= 4 probes it held the spectrum of every graph
 *                       tested, from M = 3 on), or
 *   DOS_BOUND_RITZ      r = beta_M |s_M|, the residual of the Ritz pair (s_M
 *                       the last component of the tridiagonal's unit
 *                       eigenvector): tight once the extreme Ritz values have
 *                       converged (M >= 30, Nz >= 4), too narrow before.
 * [a, b] is the union over the probes widened by pad (b - a) at each end,
 * with ends that are eigenvalues of every graph with an edge taken exactly
 * (lambda_max(H) = 1, lambda_min(D - A) = lambda_min(I - H) = 0), clipped to
 * the Gershgorin interval.  An estimate, not a proof: pad guards the FP32
 * rounding of the Ritz values (0.01 is ample).
 *   op  DOS_OP_*;  M in [1, 4096], Nz in [1, 128];  bound DOS_BOUND_*;
 *   pad in [0, 1];  interval_out [host] double[2].
 * Synchronises `stream`.  Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_spectral_interval(dos_graph_t g, int op, int M, int Nz, uint64_t seed,
                          int bound, double pad, double* interval_out,
                          void* stream);

/* The Gauss rule of each probe (§3.2): nodes_out[p * M + i] = eigenvalue tau_i
 * of Gamma_M (ascending), weights_out[p * M + i] = |p_i1|^2 (Christoffel
 * numbers; they sum to 1); slots past steps[p] hold 0.  Inputs as produced
 * by dos_lanczos [device].  Stream-ordered.  Errors: DOS_EINVAL. */
int dos_gauss_rules(const double* alpha, const double* beta,
                    const int32_t* steps, int M, int Nz, double* nodes_out,
                    double* weights_out, void* stream);

/* §3.2 (Gauss rule), Eq. (9). Chebyshev moments of the probe-averaged Gauss
 * rules, d_out[m] = (1/Nz) sum_p e_1^T T_m(Gamma_p) e_1, m < m_count [device
 * double[m_count]]; equal to the KPM moments of the same probes for m <= 2
 * steps - 1 (Gauss exactness).  Stream-ordered.  Errors: DOS_EINVAL,
 * DOS_ENOMEM. */
int dos_gql_moments(const double* alpha, const double* beta,
                    const int32_t* steps, int M, int Nz, int m_count,
                    double* d_out, void* stream);

/* §3.2, §4.1 (histogram). GQL density: bin masses of the rules' point masses
 * averaged over probes, hist_out [device] double[n_bins] over n_bins equal
 * bins of [-1, 1] (a node within 1e-9 of an interior edge splits evenly).
 * Stream-ordered. Errors: DOS_EINVAL. */
int dos_gql_histogram(const double* nodes, const double* weights, int M,
                      int Nz, int n_bins, double* hist_out, void* stream);

/* ---------------------------------------------------------------------
 * Traces and diagonals of matrix functions (§6: centralities and
 * connectivity indices such as the Estrada index are traces and diagonals
 * of f(X)).  With X~ = (X - c) / r on [a, b] -> [-1, 1] (Eq. (5)) and
 * f(c + r x) = sum_m g_m T_m(x):
 *   tr f(X) = N sum_m g_m d_m (+ f(0) per node without edges),
 *   f(X)_kk = sum_m g_m T_m(X~)_kk, estimated from LDOS moments (Eq. (10),
 *   (12)).  Estrada index: tr exp(A); subgraph centrality: exp(A)_kk;
 *   resolvent centrality: ((I - p A)^{-1})_kk; heat kernel: exp(-t L).
 * --------------------------------------------------------------------- */

/* Functions of dos_fn_coeffs. */
enum {
  DOS_FN_EXP = 0,       /* f(x) = exp(p x) */
  DOS_FN_RESOLVENT = 1  /* f(x) = 1 / (1 - p x); 1 - p x must not vanish on [lo, hi] */
};

/* §6, Eq. (5) (Chebyshev expansion of f on [a, b]). Chebyshev coefficients of
 * f on [lo, hi]: coef_out [device double[M]] with f(c + r x) ~ sum_m
 * coef_out[m] T_m(x), by interpolation at max(4M, 256) Chebyshev-Gauss points.
 * Stream-ordered.  Errors: DOS_EINVAL (unknown fn, lo >= hi, M outside [1,
 * 2^20], a resolvent pole inside [lo, hi]). */
int dos_fn_coeffs(int fn, double p, double lo, double hi, int M,
                  double* coef_out, void* stream);

/* §6, Eq. (9), (11) (trace from moments). tr f(X): out [device double[1]] = N
 * sum_m coef[m] d[m] + (nodes without edges) x f(0), f(0) = 1 for both
 * functions; d [device double[M]] DOS moments of X~ on the same interval as
 * coef (dos_moments_op), N the graph's nodes with edges.  Stream-ordered.
 * Errors: DOS_EINVAL. */
int dos_fn_trace(dos_graph_t g, const double* coef, const double* d, int M,
                 double* out, void* stream);

/* §6, Eq. (10), (12) (diagonal from LDOS moments). f(X)_kk for every node:
 * out[k] [device double[N]] = sum_m coef[m] C[m][k] over the moment-major LDOS
 * matrix C [device float[M * N]] of ldos_moments_op (compact node ids).  FP32
 * products and sums of coef / max|coef|, the scale applied in FP64 (no
 * overflow for large f).  HBM-bound: reads M N 4 bytes. Stream-ordered.
 * Errors: DOS_EINVAL. */
int dos_fn_diag(const float* C, int64_t N, int M, const double* coef,
                double* out, void* stream);

/* ---------------------------------------------------------------------
 * Batches of graphs (one operator for many small graphs).
 * --------------------------------------------------------------------- */

/*
 * dos_build_csr_batched -- a batch of graphs as one operator.
 * Graph g owns the original node ids [node_offset[g], node_offset[g+1]);
 * src/dst (as for dos_build_csr, global ids) must only join nodes of the same
 * graph.  The batch's normalized adjacency is the block-diagonal union of the
 * graphs' (§2.1), so its spectrum is the union of theirs and the step
 * kernels advance every graph at once.
 *   node_offset [host] int64[n_graphs+1], node_offset[0] = 0, non-decreasing.
 * The handle works with every single-graph call (as the union) and with
 * dos_moments_batched.  Synchronises `stream`.
 * Errors: DOS_EINVAL (an edge between two graphs, bad offsets), as
 * dos_build_csr otherwise.
 */
int dos_build_csr_batched(const int64_t* src, const int64_t* dst,
                          int64_t n_edges, const int64_t* node_offset,
                          int64_t n_graphs, uint32_t flags, void* stream,
                          dos_graph_t* out);

/* Batches: a project addition (§2.1 per graph). Batch sizes [host outputs; any
 * may be NULL]: n_graphs (0 for a graph from dos_build_csr), and per graph its
 * non-isolated node count graph_n[n_graphs] and isolated node count
 * graph_isolated[n_graphs]. */
int dos_batch_info(dos_graph_t g, int64_t* n_graphs, int64_t* graph_n,
                   int64_t* graph_isolated);

/*
 * dos_moments_batched -- DOS moments of every graph of a batch.
 * Paper: §3.1, Eq. (6), (9), (11), per graph (the union's Chebyshev
 * recurrence restricted to a graph's block is that graph's recurrence).
 *   d_out [device] double[n_graphs * M]: d_out[g * M + m] = d_m of graph g,
 *         normalised by its non-isolated node count times Nz (NaN for a graph
 *         without edges).  Same probes as dos_moments keyed by global ids.
 *   M >= 2.  No filter.
 * The sequence of kernels is captured into a CUDA graph on the first call
 * with a given (M, Nz, seed, prec, d_out, plan), kept on the handle, and
 * replayed with one graph launch on `stream` by later calls.  The per-graph
 * FP64 accumulation uses atomics, so the last bits of the moments may vary
 * from run to run.  Stream-ordered.
 * Errors: DOS_EINVAL (not a batch, M < 2, ...), DOS_ENOMEM, DOS_ECUDA.
 */
int dos_moments_batched(dos_graph_t g, int M, int Nz, uint64_t seed, int prec,
                        double* d_out, void* stream);

/*
 * A project addition (tuning of the §3.1 step).
 * dos_autotune -- time the step kernel's candidate plans (probe tile widths
 * with at most 16 tiles, 1 to 3 light-row CTAs per SM) on this graph for
 * (Nz, prec) and keep the fastest on the handle; later dos_moments /
 * ldos_moments / dos_moments_batched calls with the same Nz and prec use it
 * unless dos_set_plan forces another.  Outputs [host, may be NULL] the chosen
 * tile width and CTAs per SM.  Synchronises `stream`.
 */
int dos_autotune(dos_graph_t g, int Nz, int prec, void* stream,
                 int* tile_width, int* ctas_per_sm);

/*
 * dos_density_batched -- dos_density (kernel, no scale, no spikes) for every
 * graph of a batch: hist_out[g * n_bins + b] from d[g * M .. g * M + M).
 * Paper: §2.2 spectral histogram, Eq. (7)-(8); §4.1 Jackson damping.
 *   d        [device] double[n_graphs * M] (e.g. from dos_moments_batched)
 *   hist_out [device] double[n_graphs * n_bins]
 * Errors: DOS_EINVAL (null pointer, M or n_bins outside [1, 2^20],
 * n_graphs < 1).  Stream-ordered.
 */
int dos_density_batched(const double* d, int M, int64_t n_graphs, int n_bins,
                        int kernel, double* hist_out, void* stream);

/* ---------------------------------------------------------------------
 * Learned reconstruction of the density from few noisy moments.
 *
 * Not part of the paper: a small fully connected network (ReLU hidden layers,
 * softmax output over n_bins histogram bins) that maps a graph's feature
 * vector (the Jackson histogram and the first K moments of a cheap KPM run)
 * to its spectral histogram, trained with softmax cross-entropy against the
 * histograms of an accurate KPM run and Adam (Kingma & Ba, 2015;
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected).  Plain Jackson
 * KPM (dos_density) is its fallback.
 *
 * Parameters are one flat float32 buffer: for each layer l, W_l (out_l x
 * in_l, row-major) then b_l[out_l].  All matrices are row-major float32 on
 * the device.  Every call is stream-ordered; its reductions run in a fixed
 * order, so results are bit-reproducible.
 * --------------------------------------------------------------------- */

/* Learned reconstruction: a project addition, not in the paper. Network with
 * n_layers weight layers of sizes[0] -> sizes[1] -> ... -> sizes[n_layers]
 * (each in [1, 8192], n_layers in [1, 16]); weights He-uniform from
 * SplitMix64(seed), biases 0.  Synchronises the device. Errors: DOS_EINVAL,
 * DOS_ENOMEM. */
int dos_mlp_create(int n_layers, const int* sizes, uint64_t seed,
                   dos_mlp_t* out);
void dos_mlp_destroy(dos_mlp_t net);
/* Project addition (learned reconstruction). Number of float32 parameters
 * [host output]. */
int dos_mlp_param_count(dos_mlp_t net, int64_t* count);
/* Project addition (learned reconstruction). Copy the parameters to / from a
 * device buffer of dos_mlp_param_count floats.  set_params also resets Adam's
 * moments and step count. */
int dos_mlp_get_params(dos_mlp_t net, float* out, void* stream);
int dos_mlp_set_params(dos_mlp_t net, const float* in, void* stream);
/* Project addition (learned reconstruction): checkpoint and resume of
 * training.  get_state copies the parameters and Adam's first and second
 * moments (each a device buffer of dos_mlp_param_count floats, or NULL to
 * skip it) and the number of Adam steps taken; set_state loads all of them,
 * so that training continues exactly as if it had not been interrupted.
 * Errors: DOS_EINVAL (null handle or buffer, step outside [0, 2^31 - 1]). */
int dos_mlp_get_state(dos_mlp_t net, float* params, float* m, float* v,
                      int64_t* step, void* stream);
int dos_mlp_set_state(dos_mlp_t net, const float* params, const float* m,
                      const float* v, int64_t step, void* stream);

/* Project addition (learned reconstruction). probs[rows][sizes[n_layers]] =
 * softmax(network(x)), x[rows][sizes[0]]. Errors: DOS_EINVAL (rows < 1, null
 * pointer), DOS_ENOMEM. */
int dos_mlp_forward(dos_mlp_t net, const float* x, int rows, float* probs,
                    void* stream);

/* Project addition (learned reconstruction). Cross-entropy -(1/rows) sum t log
 * p of targets t[rows][out] (rows of t sum to 1) and its gradient.  loss
 * [device] float[1] or NULL; grad [device] float[param_count] or NULL (the
 * gradient is kept on the handle). */
int dos_mlp_loss_grad(dos_mlp_t net, const float* x, const float* t, int rows,
                      float* loss, float* grad, void* stream);

/* Project addition (learned reconstruction). One Adam step on the minibatch
 * rows idx[0..rows) of (x, t) (idx [device] int32, NULL = the first `rows`
 * rows) with learning rate lr > 0; loss [device] float[1] or NULL receives the
 * minibatch loss before the step. */
int dos_mlp_train_step(dos_mlp_t net, const float* x, const float* t,
                       const int32_t* idx, int rows, float lr, float* loss,
                       void* stream);

/* Project addition (learned reconstruction; inputs from §3.1, §4.1).
 * Feature rows for the network, one per graph g < n_graphs:
 *   x_out[g] = [ n_bins * hist[g * n_bins + b] for b < n_bins,
 *                d[g * ld_d + m] for 1 <= m < K,
 *                and, when stats is not NULL, with (mu1, mu2, dmax, e) =
 *                stats[4 g .. 4 g + 3] as dos_graph_stats returns them:
 *                log(mu1) / 10, (log(mu2) / 2 - log(mu1)) / 10,
 *                log(dmax) / 10, log(e) / 10 ]
 * (n_bins + K - 1, plus 4 with stats, floats per row).  hist [device]
 * double (a Jackson histogram, e.g. dos_density_batched), d [device] double
 * moments (row stride ld_d >= K), stats [device] double[4 n_graphs] or NULL.
 * Errors: DOS_EINVAL. */
int dos_mlp_features(const double* hist, int n_bins, const double* d,
                     int ld_d, int K, const double* stats, int64_t n_graphs,
                     float* x_out, void* stream);

/* Project addition (learned reconstruction: the network's degree inputs).
 * Degree statistics of a graph's non-isolated nodes and its noise level:
 * stats_out [device] double[4] = (mean degree, mean squared degree, largest
 * degree, N * Nz); the sums are exact (64-bit integers).  Stream-ordered.
 * Errors: DOS_EINVAL. */
int dos_graph_stats(dos_graph_t g, int Nz, double* stats_out, void* stream);

/* Density from the network's output: hist_out[r][b] = scale * probs[r][b]
 * plus point masses (lambda, mass) pairs in `spikes` [host, n_spikes <= 64],
 * placed as by dos_density (a point within 1e-9 of an interior bin edge
 * splits evenly).  With a twin filter, scale = r / N and one spike at 0 of
 * mass (removed + isolated) / N, as for the filtered series (§3.4).
 *   probs [device] float[rows][n_bins]; hist_out [device] double[rows][n_bins].
 * Errors: DOS_EINVAL. */
int dos_hist_assemble(const float* probs, int n_bins, int64_t rows,
                      double scale, const double* spikes, int n_spikes,
                      double* hist_out, void* stream);

/* Project addition (learned reconstruction; §4.1 histograms). Training
 * targets: t_out[g][b] = max(hist[g][b], 0) / sum_b max(hist[g][b], 0)
 * (uniform if that sum is 0).  Errors: DOS_EINVAL. */
int dos_hist_normalize(const double* hist, int n_bins, int64_t n_graphs,
                       float* t_out, void* stream);

/* ---------------------------------------------------------------------
 * Tuning and instrumentation (not part of the method).
 * --------------------------------------------------------------------- */

/* Tuning of the §3.1 step, not in the paper. Planner override (tuning): force
 * the probe tile width t (a power of two in [4, 64] that is a multiple of 16
 * bytes of the storage type; 0 = automatic) and the resident CTAs per SM of
 * the light-row step kernel (0 = as many as fit) of later dos_moments /
 * ldos_moments calls.  Process-wide. Errors: DOS_EINVAL. */
int dos_set_plan(int tile_width, int ctas_per_sm);

/* Tuning of the §3.1 step, not in the paper. The plan dos_moments would use
 * for (g, Nz, prec): tile width t, light-row CTAs per SM, number of tiles T =
 * ceil(Nz / t) and the number of CTAs of the light-row kernel [host outputs;
 * any may be NULL]. */
int dos_get_plan(dos_graph_t g, int Nz, int prec, int* tile_width,
                 int* ctas_per_sm, int* tiles, int* grid_x);

/* Failure detection, not in the paper. Status of the device-side error word of
 * the current device.  A kernel that gives up on a bounded wait records it
 * there, and the moments of a call that saw a non-zero word are NaN.  The
 * current step kernels stage their data with cp.async groups and wait with
 * cp.async.wait_group only (no spin on a flag or an mbarrier), so no kernel
 * of this library writes the word; it is kept for the ABI.  Synchronises
 * `stream`, returns the word in *status (0 = none; may be NULL) and clears
 * it.  Returns DOS_ETIMEOUT if the word was set, else DOS_OK. */
int dos_device_status(void* stream, int* status);

/* Instrumentation, not in the paper. Number of kernels this library has
 * launched since load (all threads). */
int64_t dos_launch_count(void);

/* Test hook, not in the paper (failure detection without a GPU fault).
 * after >= 0: the library's device allocations succeed `after` more times and
 * the next one fails as an out-of-memory cudaMalloc would (the call that made
 * it returns DOS_ENOMEM, "injected allocation failure" in dos_last_error);
 * the hook then disarms itself.  after < 0 disarms it.  Process-wide; device
 * memory that torch or the caller allocates is not affected. */
int dos_test_fail_alloc(int64_t after);

/* Instrumentation, not in the paper. Enable (1) / disable (0) CUDA-event
 * timing of the Chebyshev step kernels. While enabled, every step launch is
 * bracketed by events on its own stream. */
int dos_profile_enable(int on);

/* Instrumentation, not in the paper. Total device time (ms) and launch count
 * of the step kernels recorded since the last reset; synchronises on the
 * recorded events.  reset != 0 clears. */
int dos_profile_read(double* total_ms, int64_t* launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* NETDOS_H */
