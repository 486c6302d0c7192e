/*
 * netgen_core.h -- per-synapse draws of the seeded synthetic voxel network.
 *
 * This is the INPUT GENERATOR, shared by the CPU oracle's inputs and the GPU
 * library's inputs.  It holds none of the simulated method's arithmetic: it
 * only decides who connects to whom and with which stored weight.
 *
 * Structure (paper section III.B and Table I): voxels of heterogeneous size,
 * the first floor(0.8 n_v) neurons of each voxel excitatory, fixed in-degree K
 * per neuron (section V.D's connection tables), presynaptic partners drawn
 * with replacement (multiple edges allowed), no self loops; inputs k <
 * K_intra come from the neuron's own voxel, the rest from other voxels chosen
 * by a row-normalised DTI-like matrix and are excitatory only (long-range
 * connections are excitatory, section III.B).
 *
 * Every draw is a word of Philox4x32-10 (Salmon et al. 2011) at counter
 * {i_lo, i_hi, k, DG_TAG_SYN} under the network key, mapped to integers by
 * 32x32->64 multiply-high and by integer thresholds, so host and device give
 * identical bits.
 */
#ifndef DTB_NETGEN_CORE_H
#define DTB_NETGEN_CORE_H
#include <stdint.h>

#ifdef __CUDACC__
#define DG_HD __host__ __device__ __forceinline__
#else
#define DG_HD static inline
#endif

#define DG_TAG_SYN 0x53594Eu /* "SYN" */
#define DG_WBITS 12          /* weight quantile bins: 4096 */

typedef struct dg_net {
  int64_t n;              /* neurons */
  int32_t nv;             /* voxels */
  int32_t K;              /* in-degree */
  int32_t K_intra;        /* inputs 0..K_intra-1 come from the neuron's own voxel */
  int32_t pad_;
  const int64_t* vstart;  /* [nv+1] */
  const int64_t* nexc;    /* [nv] excitatory neurons of each voxel (its first nexc[v]) */
  const int64_t* dti_ptr; /* [nv+1] row v lists the source voxels of target voxel v */
  const int32_t* dti_src; /* source voxel ids */
  const uint64_t* dti_cum;/* cumulative row probabilities times 2^32; the last of a row is 2^32 */
  uint32_t key0, key1;
} dg_net;

DG_HD void dg_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                     uint32_t out[4]) {
  for (int r = 0; r < 10; r++) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t h1 = (uint32_t)(p1 >> 32), h0 = (uint32_t)(p0 >> 32);
    c0 = h1 ^ c1 ^ k0;
    c1 = (uint32_t)p1;
    c2 = h0 ^ c3 ^ k1;
    c3 = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Input k of neuron i (in voxel vt): presynaptic id, class (0 = E, 1 = I) and
 * weight-quantile bin. */
DG_HD void dg_synapse(const dg_net* g, int64_t i, int32_t vt, int32_t k, int32_t* pre, int32_t* cls,
                      uint32_t* wbin) {
  uint32_t r[4];
  dg_philox((uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)k, DG_TAG_SYN, g->key0, g->key1, r);
  const int64_t s0 = g->vstart[vt];
  const int64_t nvt = g->vstart[vt + 1] - s0;
  const int64_t b0 = g->dti_ptr[vt], b1 = g->dti_ptr[vt + 1];
  if (k < g->K_intra || b1 == b0) {
    int64_t loc = (int64_t)(((uint64_t)r[0] * (uint64_t)(nvt - 1)) >> 32);
    if (loc >= i - s0) loc++;
    *pre = (int32_t)(s0 + loc);
    *cls = loc < g->nexc[vt] ? 0 : 1;
  } else {
    int64_t lo = b0, hi = b1 - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((uint64_t)r[1] < g->dti_cum[mid]) hi = mid; else lo = mid + 1;
    }
    const int32_t vs = g->dti_src[lo];
    *pre = (int32_t)(g->vstart[vs] + (int64_t)(((uint64_t)r[2] * (uint64_t)g->nexc[vs]) >> 32));
    *cls = 0;
  }
  *wbin = r[3] >> (32 - DG_WBITS);
}

#endif
