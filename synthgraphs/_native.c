/* Native helpers of the synthetic graph generators (plain C, no method
 * arithmetic).  Random draws come from SplitMix64 (Steele, Lea, Flood 2014)
 * seeded by the caller, so the output is the same on every machine. */
#include <stdint.h>

static uint64_t sm_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform integer in [0, n) by the multiply-high method (Lemire 2019) */
static uint64_t sm_below(uint64_t* state, uint64_t n) {
  return (uint64_t)(((unsigned __int128)sm_next(state) * n) >> 64);
}

/* Barabasi-Albert: seed clique K_{m+1}, then every node t > m attaches to m
 * distinct earlier nodes drawn with probability proportional to degree
 * (uniform draws from the list of edge endpoints, repeats redrawn).
 * ends: scratch of 2 * n_edges int64; src/dst: n_edges each, where
 * n_edges = m(m+1)/2 + (n - m - 1) m.  Returns the number of edges written. */
int64_t ba_edges(int64_t n, int64_t m, uint64_t seed, int64_t* src, int64_t* dst, int64_t* ends) {
  uint64_t st = seed;
  int64_t e = 0, n_ends = 0;
  for (int64_t a = 0; a <= m; ++a)
    for (int64_t b = a + 1; b <= m; ++b) {
      src[e] = a;
      dst[e] = b;
      ends[n_ends++] = a;
      ends[n_ends++] = b;
      ++e;
    }
  int64_t chosen[64];
  for (int64_t t = m + 1; t < n; ++t) {
    int64_t k = 0;
    while (k < m) {
      const int64_t c = ends[sm_below(&st, (uint64_t)n_ends)];
      int dup = 0;
      for (int64_t i = 0; i < k; ++i) dup |= chosen[i] == c;
      if (!dup) chosen[k++] = c;
    }
    for (int64_t i = 0; i < m; ++i) {
      src[e] = t;
      dst[e] = chosen[i];
      ends[n_ends++] = t;
      ends[n_ends++] = chosen[i];
      ++e;
    }
  }
  return e;
}
