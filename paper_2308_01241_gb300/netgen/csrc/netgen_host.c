/*
 * netgen_host.c -- host side of the seeded synthetic network generator
 * (input generator; see netgen_core.h).  Builds the pull form (connection
 * tables of paper section V.D) for any range of postsynaptic neurons and
 * turns a pull form into an outgoing CSR by a stable counting sort.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "netgen_core.h"

static int32_t voxel_of(const dg_net* g, int64_t i) {
  int32_t lo = 0, hi = g->nv - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (g->vstart[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

/* Pull form of neurons [i0, i1): pre, cls, wbin are [(i1 - i0) * K]. */
int dg_host_pull(const dg_net* g, int64_t i0, int64_t i1, int32_t* pre, uint8_t* cls, uint16_t* wbin) {
  if (i0 < 0 || i1 > g->n || i0 > i1) return -1;
  for (int64_t i = i0; i < i1; i++) {
    const int32_t vt = voxel_of(g, i);
    for (int32_t k = 0; k < g->K; k++) {
      int32_t p, c;
      uint32_t b;
      dg_synapse(g, i, vt, k, &p, &c, &b);
      const int64_t e = (i - i0) * (int64_t)g->K + k;
      pre[e] = p;
      cls[e] = (uint8_t)c;
      wbin[e] = (uint16_t)b;
    }
  }
  return 0;
}

/* Outgoing CSR from a pull form: rows by presynaptic neuron, entries in
 * ascending (postsynaptic, input) order.  word = target | class << 30. */
int dg_host_transpose(int64_t n, int32_t K, const int32_t* pre, const uint8_t* cls, const uint16_t* wbin,
                      int64_t* row_ptr, uint32_t* word, uint16_t* wbin_out) {
  if (n < 0 || K < 0) return -1;
  memset(row_ptr, 0, (size_t)(n + 1) * sizeof(int64_t));
  const int64_t nnz = n * (int64_t)K;
  for (int64_t e = 0; e < nnz; e++) {
    if (pre[e] < 0 || pre[e] >= n) return -1;
    row_ptr[pre[e] + 1]++;
  }
  for (int64_t i = 0; i < n; i++) row_ptr[i + 1] += row_ptr[i];
  int64_t* fill = (int64_t*)calloc((size_t)(n ? n : 1), sizeof(int64_t));
  if (!fill) return -2;
  for (int64_t i = 0; i < n; i++)
    for (int32_t k = 0; k < K; k++) {
      const int64_t e = i * (int64_t)K + k;
      const int32_t p = pre[e];
      const int64_t q = row_ptr[p] + fill[p]++;
      word[q] = (uint32_t)i | ((uint32_t)cls[e] << 30);
      wbin_out[q] = wbin[e];
    }
  free(fill);
  return 0;
}
